"""Thin Python binding of the C ABI in include/glemur.h (argument marshalling
only; every step of the relaxation runs in the CUDA library).

Fields are float64 arrays of shape (3, nz, ny, nx): a CUDA torch tensor is
passed as a device pointer, a numpy array (or CPU tensor) as a host pointer.
PyTorch supplies the device workspace and the stream; the library allocates
nothing.  There is no CPU fallback: without the compiled library every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERR = {-1: "BADARG", -2: "CUDA", -3: "COLLAPSED", -4: "NONFINITE", -5: "DT_UNDERFLOW",
       -6: "WORKSPACE", -7: "TOO_LARGE", -8: "TIMEOUT"}
FP64, MIXED = 0, 1
MIMETIC, DIRECT, NNN = 0, 1, 2
MEM_DEVICE, MEM_HOST = 0, 1


class GlemurError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {ERR.get(code, code)} ({code})")


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("curl", C.c_int), ("lambda0", C.c_double),
                ("dt0", C.c_double), ("dt_min", C.c_double), ("grow_max", C.c_double),
                ("shrink_min", C.c_double), ("max_rejects", C.c_int),
                ("diag_each_attempt", C.c_int), ("safety", C.c_double),
                ("periodic_z", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("accepted", C.c_longlong), ("rejected", C.c_longlong), ("t", C.c_double),
                ("dt", C.c_double), ("lambda_", C.c_double), ("energy", C.c_double),
                ("xi", C.c_double), ("xi_sin", C.c_double), ("status", C.c_int),
                ("dt_last", C.c_double)]

    def as_dict(self):
        return dict(accepted=self.accepted, rejected=self.rejected, t=self.t, dt=self.dt,
                    lam=self.lambda_, energy=self.energy, xi=self.xi, xi_sin=self.xi_sin,
                    status=self.status, dt_last=self.dt_last)


EXPORTS = ["glemur_default_opts", "glemur_workspace_bytes", "glemur_init_grid",
           "glemur_set_x", "glemur_set_B0", "glemur_get_x", "glemur_velocity",
           "glemur_step", "glemur_attempts", "glemur_step_fixed", "glemur_energy",
           "glemur_forcefree_err", "glemur_get_stats", "glemur_kernels_per_attempt",
           "glemur_profile_attempt", "glemur_energy_static", "glemur_destroy",
           "glemur_strerror", "glemur_adjoint_workspace_bytes", "glemur_vjp_step",
           "glemur_loss_grad", "glemur_param_contract", "glemur_state_bytes",
           "glemur_get_state", "glemur_set_state", "glemur_get_dt_schedule",
           "glemur_deviation", "glemur_alpha_line", "glemur_convexity",
           "glemur_adjoint_segment_bytes", "glemur_adjoint_segment"]
DT_LOG = 65536  # accepted step sizes the device keeps (GLEMUR_DT_LOG)
LOSS_ENERGY, LOSS_XI = 0, 1

_lib = None


def lib_path() -> str:
    return _build.LIB


def lib() -> C.CDLL:
    """Load libglemur.so (building it first when the toolkit is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    try:
        path = _build.build()
    except Exception as e:  # no toolkit: use an existing build or fail loudly
        if not os.path.exists(path):
            raise RuntimeError(f"libglemur.so is not built and cannot be built: {e}") from e
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.glemur_default_opts.argtypes = [C.POINTER(Opts)]
    L.glemur_default_opts.restype = None
    L.glemur_workspace_bytes.argtypes = [ip, ip, ip, ip]
    L.glemur_workspace_bytes.restype = C.c_size_t
    L.glemur_init_grid.argtypes = [C.POINTER(vp), ip, ip, ip, dp, dp, C.POINTER(Opts), vp, vp,
                                   C.c_size_t]
    L.glemur_set_x.argtypes = [vp, vp, ip]
    L.glemur_set_B0.argtypes = [vp, vp, ip]
    L.glemur_get_x.argtypes = [vp, vp, ip]
    L.glemur_velocity.argtypes = [vp, vp, ip]
    L.glemur_step.argtypes = [vp, ip, C.POINTER(Stats)]
    L.glemur_attempts.argtypes = [vp, ip]
    L.glemur_step_fixed.argtypes = [vp, C.c_double, C.POINTER(Stats)]
    L.glemur_energy.argtypes = [vp, dp]
    L.glemur_forcefree_err.argtypes = [vp, dp, dp]
    L.glemur_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.glemur_get_dt_schedule.argtypes = [vp, C.c_longlong, ip, dp]
    L.glemur_deviation.argtypes = [vp, vp, vp, dp, dp]
    L.glemur_alpha_line.argtypes = [vp, ip, ip, C.c_double, dp, dp]
    L.glemur_convexity.argtypes = [vp, C.POINTER(C.c_longlong), vp]
    L.glemur_kernels_per_attempt.argtypes = [vp]
    L.glemur_profile_attempt.argtypes = [vp, C.POINTER(C.c_float), ip]
    L.glemur_energy_static.argtypes = [ip, ip, ip, dp, dp, vp, vp, vp, vp]
    L.glemur_adjoint_workspace_bytes.argtypes = [ip, ip, ip, ip]
    L.glemur_adjoint_workspace_bytes.restype = C.c_size_t
    L.glemur_vjp_step.argtypes = [vp, C.c_double, vp, vp, vp, vp, C.c_size_t]
    L.glemur_loss_grad.argtypes = [vp, ip, dp, vp, vp, vp, C.c_size_t]
    L.glemur_param_contract.argtypes = [ip, C.c_longlong, vp, vp, vp, vp]
    L.glemur_adjoint_segment_bytes.argtypes = [vp, ip, ip]
    L.glemur_adjoint_segment_bytes.restype = C.c_size_t
    L.glemur_adjoint_segment.argtypes = [vp, vp, dp, ip, ip, ip, dp, vp, vp, vp, C.c_size_t, vp,
                                         C.c_size_t]
    L.glemur_state_bytes.argtypes = [vp]
    L.glemur_state_bytes.restype = C.c_size_t
    L.glemur_get_state.argtypes = [vp, vp]
    L.glemur_set_state.argtypes = [vp, vp]
    L.glemur_destroy.argtypes = [vp]
    L.glemur_destroy.restype = None
    L.glemur_strerror.argtypes = [ip]
    L.glemur_strerror.restype = C.c_char_p
    _lib = L
    return L


def _check(rc, what):
    if rc != OK:
        raise GlemurError(rc, what)


def default_opts() -> Opts:
    o = Opts()
    lib().glemur_default_opts(C.byref(o))
    return o


def workspace_bytes(nx, ny, nz, precision=FP64) -> int:
    return int(lib().glemur_workspace_bytes(nx, ny, nz, precision))


def _field_ptr(a, shape, writable=False):
    """(pointer, mem kind, keep-alive) of a float64 (3, nz, ny, nx) field."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if tuple(a.shape) != shape or a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError(f"expected contiguous float64 tensor of shape {shape}")
            return (a.data_ptr(), MEM_DEVICE if a.is_cuda else MEM_HOST, a)
    except ImportError:
        pass
    arr = np.asarray(a)
    if arr.shape != shape or arr.dtype != np.float64 or not arr.flags.c_contiguous:
        if writable:
            raise ValueError(f"expected C-contiguous float64 array of shape {shape}")
        arr = np.ascontiguousarray(arr, dtype=np.float64).reshape(shape)
    return (arr.ctypes.data, MEM_HOST, arr)


class Relaxation:
    """A grid of nx*ny*nz nodes with labels on [lo, hi] and its relaxation
    state, bound to one CUDA device and stream (glemur_init_grid)."""

    def __init__(self, nx, ny, nz, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                 precision=FP64, curl=MIMETIC, lambda0=None, dt0=None, dt_min=None,
                 grow_max=None, shrink_min=None, max_rejects=None, diag_each_attempt=None,
                 safety=None, periodic_z=None, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the GB300 relaxation library needs a CUDA device")
        self.shape = (3, nz, ny, nx)
        self.dims = (nx, ny, nz)
        self.device = torch.device(device if device is not None else "cuda")
        o = default_opts()
        o.precision, o.curl = int(precision), int(curl)
        for name, v in (("lambda0", lambda0), ("dt0", dt0), ("dt_min", dt_min),
                        ("grow_max", grow_max), ("shrink_min", shrink_min),
                        ("max_rejects", max_rejects), ("diag_each_attempt", diag_each_attempt),
                        ("safety", safety), ("periodic_z", periodic_z)):
            if v is not None:
                setattr(o, name, type(getattr(o, name))(v))
        self.opts = o
        L = lib()
        nbytes = L.glemur_workspace_bytes(nx, ny, nz, o.precision)
        if nbytes == 0:
            raise GlemurError(-1, "glemur_workspace_bytes")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            lo_a = (C.c_double * 3)(*lo)
            hi_a = (C.c_double * 3)(*hi)
            h = C.c_void_p()
            rc = L.glemur_init_grid(C.byref(h), nx, ny, nz, lo_a, hi_a, C.byref(o),
                                    C.c_void_p(self.stream.cuda_stream),
                                    C.c_void_p(self.workspace.data_ptr()), int(nbytes))
        _check(rc, "glemur_init_grid")
        self._h = h
        self._held = []  # (event, host buffer) pairs the stream may still read

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.glemur_destroy(h)
            self._h = None

    # -- fields -----------------------------------------------------------
    def set_x(self, x, non_blocking=False):
        """Positions x (3, nz, ny, nx) float64, on the device or the host.
        A host buffer is read asynchronously; with non_blocking=False the
        call waits for the copy, with non_blocking=True (as torch's
        Tensor.to) it returns at once and the caller must not modify the
        buffer until the stream has passed the copy (the library keeps it
        alive until then)."""
        p, mem, keep = _field_ptr(x, self.shape)
        _check(lib().glemur_set_x(self._h, p, mem), "glemur_set_x")
        self._after_host_read(mem, keep, non_blocking)

    def set_B0(self, B0, non_blocking=False):
        """B0 (3, nz, ny, nx) float64 at the label grid; host buffers as in
        set_x."""
        p, mem, keep = _field_ptr(B0, self.shape)
        _check(lib().glemur_set_B0(self._h, p, mem), "glemur_set_B0")
        self._after_host_read(mem, keep, non_blocking)

    def _after_host_read(self, mem, keep, non_blocking):
        if mem != MEM_HOST:
            return
        if not non_blocking:
            self.stream.synchronize()
            return
        import torch
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self._held = [(e, k) for e, k in self._held if not e.query()]
        self._held.append((ev, keep))

    def get_x(self, out=None):
        """Current positions: into `out` (CUDA tensor or numpy array), else a
        new CUDA tensor."""
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        p, mem, keep = _field_ptr(out, self.shape, writable=True)
        _check(lib().glemur_get_x(self._h, p, mem), "glemur_get_x")
        return out

    def velocity(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        p, mem, keep = _field_ptr(out, self.shape, writable=True)
        _check(lib().glemur_velocity(self._h, p, mem), "glemur_velocity")
        return out

    # -- stepping ---------------------------------------------------------
    def step(self, n_accept=1, check=True):
        st = Stats()
        rc = lib().glemur_step(self._h, int(n_accept), C.byref(st))
        if check:
            _check(rc, "glemur_step")
        return st.as_dict()

    def attempts(self, n):
        _check(lib().glemur_attempts(self._h, int(n)), "glemur_attempts")

    def step_fixed(self, dt, check=True):
        st = Stats()
        rc = lib().glemur_step_fixed(self._h, float(dt), C.byref(st))
        if check:
            _check(rc, "glemur_step_fixed")
        return st.as_dict()

    def dt_schedule(self, first, count):
        """Sizes of accepted steps first .. first+count-1 since set_x, as
        recorded on the device by the step control (numpy float64)."""
        out = np.empty(int(count), dtype=np.float64)
        _check(lib().glemur_get_dt_schedule(self._h, int(first), int(count),
                                            out.ctypes.data_as(C.POINTER(C.c_double))),
               "glemur_get_dt_schedule")
        return out

    def stats(self):
        st = Stats()
        _check(lib().glemur_get_stats(self._h, C.byref(st)), "glemur_get_stats")
        return st.as_dict()

    # -- diagnostics ------------------------------------------------------
    def energy(self):
        e = C.c_double()
        _check(lib().glemur_energy(self._h, C.byref(e)), "glemur_energy")
        return e.value

    def forcefree_err(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().glemur_forcefree_err(self._h, C.byref(a), C.byref(b)),
               "glemur_forcefree_err")
        return a.value, b.value

    def deviation(self, x_ref, B_ref):
        """(sigma_x, sigma_B) of the current state against the CUDA float64
        fields x_ref, B_ref (e.g. a closed-form relaxed state)."""
        for t in (x_ref, B_ref):
            p, mem, _ = _field_ptr(t, self.shape)
            if mem != MEM_DEVICE:
                raise ValueError("deviation() takes CUDA float64 fields")
        a, b = C.c_double(), C.c_double()
        _check(lib().glemur_deviation(self._h, C.c_void_p(x_ref.data_ptr()),
                                      C.c_void_p(B_ref.data_ptr()), C.byref(a), C.byref(b)),
               "glemur_deviation")
        return a.value, b.value

    def alpha_line(self, i, j, a_r):
        """(alpha* along the node line (i, j, .) as a numpy array -- NaN at
        its two boundary nodes --, epsilon*)."""
        alpha = np.empty(self.dims[2], dtype=np.float64)
        e = C.c_double()
        _check(lib().glemur_alpha_line(self._h, int(i), int(j), float(a_r),
                                       alpha.ctypes.data_as(C.POINTER(C.c_double)),
                                       C.byref(e)), "glemur_alpha_line")
        return alpha, e.value

    def convexity(self, with_field=False):
        """Number of concave nodes (kappa = -1); with_field=True also returns
        kappa as an int8 CUDA tensor of shape (nz, ny, nx)."""
        import torch
        n = C.c_longlong()
        kap = None
        if with_field:
            nx, ny, nz = self.dims
            kap = torch.empty((nz, ny, nx), dtype=torch.int8, device=self.device)
        _check(lib().glemur_convexity(self._h, C.byref(n),
                                      C.c_void_p(kap.data_ptr() if kap is not None else 0)),
               "glemur_convexity")
        return (n.value, kap) if with_field else n.value

    def kernels_per_attempt(self):
        return int(lib().glemur_kernels_per_attempt(self._h))

    def profile_attempt(self):
        """One attempt with per-kernel CUDA-event durations (ms), launch order:
        stages 1..6, step control."""
        ms = (C.c_float * 16)()
        n = lib().glemur_profile_attempt(self._h, ms, 16)
        if n < 0:
            raise GlemurError(n, "glemur_profile_attempt")
        return [ms[i] for i in range(n)]

    # -- exact checkpoints ------------------------------------------------
    def get_state(self, out=None):
        """Raw state (displacement in storage precision) as a uint8 CUDA
        tensor: an exact checkpoint."""
        import torch
        n = int(lib().glemur_state_bytes(self._h))
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, device=self.device)
        _check(lib().glemur_get_state(self._h, C.c_void_p(out.data_ptr())), "glemur_get_state")
        return out

    def set_state(self, buf):
        _check(lib().glemur_set_state(self._h, C.c_void_p(buf.data_ptr())), "glemur_set_state")

    # -- adjoint ----------------------------------------------------------
    def _adj_ws(self):
        import torch
        ws = getattr(self, "_adjoint_ws", None)
        if ws is None:
            nx, ny, nz = self.dims
            n = int(lib().glemur_adjoint_workspace_bytes(nx, ny, nz, self.opts.precision))
            if n == 0:
                raise GlemurError(-1, "glemur_adjoint_workspace_bytes")
            ws = torch.empty(n, dtype=torch.uint8, device=self.device)
            self._adjoint_ws = ws
        return ws

    def vjp_step(self, dt, lam_next, lam, mu_B0):
        """lam = (dx_{n+1}/dx_n)^T lam_next, mu_B0 += (dx_{n+1}/dB0)^T lam_next
        for one step of size dt from the current state (CUDA float64 fields)."""
        ws = self._adj_ws()
        for t in (lam_next, lam, mu_B0):
            _field_ptr(t, self.shape, writable=True)
        _check(lib().glemur_vjp_step(self._h, float(dt), C.c_void_p(lam_next.data_ptr()),
                                     C.c_void_p(lam.data_ptr()), C.c_void_p(mu_B0.data_ptr()),
                                     C.c_void_p(ws.data_ptr()), ws.numel()), "glemur_vjp_step")

    def adjoint_segment(self, x0, dts, loss=LOSS_ENERGY, checkpoint_every=50):
        """glemur_adjoint_segment: the loss of the state reached from the
        positions x0 (CUDA float64 tensor) by the step sizes dts, and its
        gradients with respect to B0 and x0 -- checkpoints every
        `checkpoint_every` steps, recompute and the reverse steps, all in
        the library.  Returns (value, dL/dB0, dL/dx0)."""
        import torch
        _field_ptr(x0, self.shape)
        if not x0.is_cuda:
            raise ValueError("x0 must be a CUDA tensor")
        d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
        n, every = int(d.size), max(1, int(checkpoint_every))
        nb = int(lib().glemur_adjoint_segment_bytes(self._h, n, every))
        if nb == 0:
            raise GlemurError(-1, "glemur_adjoint_segment_bytes")
        seg = torch.empty(nb, dtype=torch.uint8, device=self.device)
        ws = self._adj_ws()
        lam = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        mu = torch.empty_like(lam)
        v = C.c_double()
        _check(lib().glemur_adjoint_segment(
            self._h, C.c_void_p(x0.data_ptr()), d.ctypes.data_as(C.POINTER(C.c_double)), n,
            every, int(loss), C.byref(v), C.c_void_p(lam.data_ptr()), C.c_void_p(mu.data_ptr()),
            C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(seg.data_ptr()), seg.numel()),
            "glemur_adjoint_segment")
        return v.value, mu, lam

    def loss_grad(self, loss, lam, mu_B0):
        """Loss of the current state; its position gradient into lam and its
        B0 gradient added to mu_B0."""
        ws = self._adj_ws()
        v = C.c_double()
        _check(lib().glemur_loss_grad(self._h, int(loss), C.byref(v), C.c_void_p(lam.data_ptr()),
                                      C.c_void_p(mu_B0.data_ptr()), C.c_void_p(ws.data_ptr()),
                                      ws.numel()), "glemur_loss_grad")
        return v.value


def param_contract(dB0, mu):
    """sum over nodes of dB0[p] . mu for each parameter p (CUDA tensors:
    dB0 (P, 3, nz, ny, nx), mu (3, nz, ny, nx)); returns a (P,) tensor."""
    import torch
    P = dB0.shape[0]
    dB0 = dB0.contiguous()
    mu = mu.contiguous()
    out = torch.empty(P, dtype=torch.float64, device=mu.device)
    _check(lib().glemur_param_contract(P, mu.numel(), C.c_void_p(dB0.data_ptr()),
                                       C.c_void_p(mu.data_ptr()), C.c_void_p(out.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream)),
           "glemur_param_contract")
    return out


def relax_with_schedule(relax, x0, n_steps):
    """Run n_steps error-controlled steps from x0 and return the accepted
    step sizes (the schedule the adjoint replays), read from the device's
    step-size log once per DT_LOG steps rather than once per step."""
    relax.set_x(x0)
    dts = []
    done = 0
    while done < n_steps:
        chunk = min(n_steps - done, DT_LOG)
        relax.step(chunk)
        dts.extend(float(v) for v in relax.dt_schedule(done, chunk))
        done += chunk
    return dts


def forward_checkpoints(relax, x0, dts, checkpoint_every=50):
    """Replay the step-size schedule `dts` from x0 (step_fixed), keeping the
    exact raw state every `checkpoint_every` steps (and at step 0): the
    forward half of the adjoint.  Leaves the relaxation at the final state."""
    every = max(1, int(checkpoint_every))
    relax.set_x(x0)
    ckpts = [relax.get_state()]
    n = len(dts)
    for i, dt in enumerate(dts):
        relax.step_fixed(dt)
        if (i + 1) % every == 0 and i + 1 < n:
            ckpts.append(relax.get_state())
    return ckpts


def reverse_sweep(relax, ckpts, dts, loss=LOSS_ENERGY, checkpoint_every=50):
    """The backward half: from checkpoints of forward_checkpoints (same
    `checkpoint_every`), recompute each segment forwards keeping its states,
    seed the loss gradient at the final state and run the steps'
    vector-Jacobian products in reverse (glemur_vjp_step).  Returns (loss
    value, dL/dB0, dL/dx0)."""
    import torch
    n = len(dts)
    every = max(1, int(checkpoint_every))
    lam = torch.zeros(relax.shape, dtype=torch.float64, device=relax.device)
    lam_next = torch.zeros_like(lam)
    mu = torch.zeros_like(lam)
    if n == 0:
        relax.set_state(ckpts[0])
        value = relax.loss_grad(loss, lam_next, mu)
        return value, mu, lam_next
    value = None
    nseg = (n + every - 1) // every
    for c in reversed(range(nseg)):
        start, end = c * every, min((c + 1) * every, n)
        relax.set_state(ckpts[c])
        states = [ckpts[c]]
        for i in range(start, end):
            relax.step_fixed(dts[i])
            states.append(relax.get_state())
        if value is None:
            relax.set_state(states[-1])
            value = relax.loss_grad(loss, lam_next, mu)
        for i in reversed(range(start, end)):
            relax.set_state(states[i - start])
            relax.vjp_step(dts[i], lam_next, lam, mu)
            lam_next, lam = lam, lam_next
        del states
    return value, mu, lam_next


def loss_and_field_gradient(relax, x0, dts, loss=LOSS_ENERGY, checkpoint_every=50):
    """Loss of the state reached from x0 by the step-size schedule `dts`
    (replayed exactly: the control law is piecewise constant in the inputs)
    and its gradient with respect to the relaxation's B0 (and to x0).

    Memory: positions are kept every `checkpoint_every` steps; the backward
    pass recomputes each segment forwards, storing its states, then runs the
    steps' vector-Jacobian products in reverse (glemur_vjp_step).
    """
    return relax.adjoint_segment(x0, dts, loss, checkpoint_every)


def _loss_value(relax, loss):
    if loss == LOSS_ENERGY:
        return relax.energy()
    return relax.forcefree_err()[0]


class RelaxationLoss:
    """torch.autograd.Function of the initial-field parameters theta: the
    loss (final E_M or xi) of the state reached from x0 by the frozen
    step-size schedule `dts`, for B0 = field(theta).

    `field(theta)` returns (B0, dB0) as CUDA float64 tensors: B0 of shape
    (3, nz, ny, nx) and its parameter derivatives dB0 of shape
    (P, 3, nz, ny, nx).  forward() only relaxes (checkpointing the state
    every `checkpoint_every` steps) and returns the loss; backward() runs the
    reverse sweep from the checkpoints and contracts the field adjoint with
    dB0 on the device (glemur_param_contract)."""

    @staticmethod
    def apply(relax, theta, field, x0, dts, loss=LOSS_ENERGY, checkpoint_every=50):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, th):
                B0, dB0 = field(th.detach())
                relax.set_B0(B0)
                ckpts = forward_checkpoints(relax, x0, dts, checkpoint_every)
                value = _loss_value(relax, loss)
                ctx.ckpts = ckpts
                ctx.dB0 = dB0
                ctx.B0 = B0
                return torch.tensor(value, dtype=torch.float64, device=th.device)

            @staticmethod
            def backward(ctx, g):
                relax.set_B0(ctx.B0)
                _, mu, _ = reverse_sweep(relax, ctx.ckpts, dts, loss, checkpoint_every)
                grad = param_contract(ctx.dB0, mu)
                ctx.ckpts = ctx.dB0 = ctx.B0 = None
                return g * grad.to(g.device)

        return _Fn.apply(theta)


class RelaxationFieldLoss:
    """torch.autograd.Function of the nodal initial field B0 itself: the
    same loss, gradient dL/dB0 (forward relaxes and checkpoints, backward
    runs the reverse sweep)."""

    @staticmethod
    def apply(relax, B0, x0, dts, loss=LOSS_ENERGY, checkpoint_every=50):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, B0_):
                relax.set_B0(B0_.detach())
                ctx.ckpts = forward_checkpoints(relax, x0, dts, checkpoint_every)
                ctx.B0 = B0_.detach()
                return torch.tensor(_loss_value(relax, loss), dtype=torch.float64,
                                    device=B0_.device)

            @staticmethod
            def backward(ctx, g):
                relax.set_B0(ctx.B0)
                _, mu, _ = reverse_sweep(relax, ctx.ckpts, dts, loss, checkpoint_every)
                ctx.ckpts = ctx.B0 = None
                return g * mu

        return _Fn.apply(B0)
