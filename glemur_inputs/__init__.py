"""Seeded synthetic workloads for the Lagrangian magneto-frictional relaxation.

This module only *describes inputs*: the logically rectangular node grid X_ijk,
the initial field B(X, 0) sampled on the nodes, and the initial grid positions
x(X, 0).  It holds none of the method's arithmetic (no Jacobian, pull-back,
curl, velocity or time stepping), so the FP64 oracle and the CUDA library can
both be driven from it without sharing any of the computation they are
compared on.

Layout of every nodal field: float64 SoA array of shape (3, nz, ny, nx);
component c of node (i, j, k) sits at [c, k, j, i].

Random numbers come from splitmix64 (Steele, Lea & Flood 2014):
    state += 0x9E3779B97F4A7C15; z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB;  r = z ^ (z >> 31)
and a uniform deviate u = (r >> 11) * 2^-53 in [0, 1).

The workloads (the paper measures on no public data set; these stand in for
the paper's analytic initial fields, section "Initial Configuration"):

* ``tube``     -- one twisted flux tube on the z axis over a uniform e_z
                  background, 16^3 nodes, x = X.
* ``braid``    -- a braid of Gaussian twist regions stacked along z with
                  alternating centres (+-0.4, 0), on a grid pre-distorted by
                  x_a = X_a + 0.05 sin(pi X_a + phi_a) with a seeded phase
                  phi_a per axis.  6 regions at 64^3 and 96^3 (amplitudes
                  +-1), 10 regions at 128^3 and 12 regions at 384^3
                  (amplitudes ~ U[-1.5, 1.5]); the 384^3 workload adds
                  0.1 x an ABC (Arnold-Beltrami-Childress) field.
* ``isohelix`` -- the paper's IsoHelix field (eq. "B init analytical").

Every B0 here is divergence-free in X: a twist region contributes
k G(r, z) (-(y - y_i), x - x_i, 0) with G depending on the distance r from its
axis only through r^2, whose divergence vanishes identically; the ABC field
is solenoidal by construction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based splitmix64 generator with the published constants."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, a: float, b: float) -> float:
        return a + (b - a) * self.uniform()


@dataclass(frozen=True)
class Grid:
    """Logically rectangular node grid: X_ijk = lo + (i h_x, j h_y, k h_z)."""

    nx: int
    ny: int
    nz: int
    lo: tuple = (-1.0, -1.0, -1.0)
    hi: tuple = (1.0, 1.0, 1.0)
    # periodic in z: planes 0 and nz-1 are ghosts of planes nz-2 and 1,
    # shifted by the period (nz - 2) h_z (section "Boundary Conditions")
    periodic_z: bool = False

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_interior(self) -> int:
        return max(self.nx - 2, 0) * max(self.ny - 2, 0) * max(self.nz - 2, 0)

    @property
    def h(self):
        n = (self.nx, self.ny, self.nz)
        return tuple((self.hi[a] - self.lo[a]) / (n[a] - 1) for a in range(3))


def nodes(g: Grid) -> np.ndarray:
    """Label coordinates X of every node, shape (3, nz, ny, nx), float64."""
    h = g.h
    xs = g.lo[0] + h[0] * np.arange(g.nx, dtype=np.float64)
    ys = g.lo[1] + h[1] * np.arange(g.ny, dtype=np.float64)
    zs = g.lo[2] + h[2] * np.arange(g.nz, dtype=np.float64)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X, Y, Z])


# ---------------------------------------------------------------- fields


def uniform_field(g: Grid, b=(0.0, 0.0, 1.0)) -> np.ndarray:
    out = np.empty((3,) + g.shape)
    for c in range(3):
        out[c] = b[c]
    return out


def twist_region(X: np.ndarray, xc: float, yc: float, zc: float, k: float,
                 l: float, L: float) -> np.ndarray:
    """k exp(-((x-xc)^2+(y-yc)^2)/l^2 - (z-zc)^2/L^2) (-(y-yc), x-xc, 0)."""
    dx = X[0] - xc
    dy = X[1] - yc
    dz = X[2] - zc
    G = k * np.exp(-(dx * dx + dy * dy) / (l * l) - dz * dz / (L * L))
    return np.stack([-dy * G, dx * G, np.zeros_like(G)])


def twist_region_grad(X, xc, yc, zc, k, l, L):
    """d/dk and d/dl of :func:`twist_region` (for parameter gradients)."""
    dx = X[0] - xc
    dy = X[1] - yc
    dz = X[2] - zc
    r2 = dx * dx + dy * dy
    E = np.exp(-r2 / (l * l) - dz * dz / (L * L))
    vec = np.stack([-dy * E, dx * E, np.zeros_like(E)])
    d_dk = vec
    d_dl = vec * (k * 2.0 * r2 / (l ** 3))
    return d_dk, d_dl


def abc_field(X: np.ndarray, A=1.0, B=1.0, C=1.0, kk=2.0 * math.pi) -> np.ndarray:
    """(A sin kz + C cos ky, B sin kx + A cos kz, C sin ky + B cos kx)."""
    x, y, z = X
    return np.stack([A * np.sin(kk * z) + C * np.cos(kk * y),
                     B * np.sin(kk * x) + A * np.cos(kk * z),
                     C * np.sin(kk * y) + B * np.cos(kk * x)])


def isohelix_field(X, B0=1.0, a_r=math.sqrt(2.0), a_z=2.0, phi=math.pi / 4):
    """Paper eq. "B init analytical" (IsoHelix)."""
    x, y, z = X
    E = np.exp(-(x * x + y * y) / a_r ** 2 - z * z / a_z ** 2)
    f = 2.0 * B0 * z / a_z ** 2 * E * phi
    return np.stack([f * y, -f * x, np.full_like(x, B0)])


# Offsets of the two Pontin09 twist regions from the mid-plane.  The paper
# does not give them; +-4 (in the IsoHelix box 8 x 8 x 20) is the value of
# {2, 3, 4, 5, 6} whose mimetic epsilon* reproduces Table 2 at n = 17 and 33,
# with n = 65 as the check.
PONTIN09_L = (4.0, -4.0)


def pontin09_field(X, phi=(math.pi / 2, -math.pi / 2), L=PONTIN09_L, B0=1.0,
                   a_r=math.sqrt(2.0), a_z=2.0):
    """Paper eq. "B init Pontin09": B0 e_z plus two twist regions at Z = L_i
    of twist angles phi_i, each 2 B0 phi_i / (pi a_r) exp(-(X^2+Y^2)/a_r^2
    - (Z-L_i)^2/a_z^2) (-Y e_x + X e_y)."""
    x, y, z = X
    Bx = np.zeros_like(x)
    By = np.zeros_like(x)
    for ph, Li in zip(phi, L):
        f = 2.0 * B0 * ph / (math.pi * a_r) * np.exp(-(x * x + y * y) / a_r ** 2
                                                    - (z - Li) ** 2 / a_z ** 2)
        Bx -= y * f
        By += x * f
    return np.stack([Bx, By, np.full_like(x, B0)])


def isohelix_relaxed(X, B0=1.0, a_r=math.sqrt(2.0), a_z=2.0, phi=math.pi / 4):
    """The IsoHelix field's exact relaxed state (eqs. "B relaxed" and "x
    analytical relaxed"): positions x_relax -- each plane Z = const turned
    about the z axis by the angle phi exp(-(X^2+Y^2)/a_r^2 - Z^2/a_z^2) --
    and the field B_relax = B0 e_z, both sampled on the nodes."""
    x, y, z = X
    th = phi * np.exp(-(x * x + y * y) / a_r ** 2 - z * z / a_z ** 2)
    c, s = np.cos(th), np.sin(th)
    xr = np.stack([c * x + s * y, c * y - s * x, z.copy()])
    Br = np.stack([np.zeros_like(x), np.zeros_like(x), np.full_like(x, B0)])
    return xr, Br


# ---------------------------------------------------------------- grids


def predistort(X: np.ndarray, seed: int, amp: float = 0.05) -> np.ndarray:
    """x_a = X_a + amp sin(pi X_a + phi_a), phi_a = 2 pi U[0,1) per axis.

    Each component depends on its own label coordinate only, so the box faces
    stay planar and dx/dX is diagonal with det >= (1 - amp pi)^3 > 0.
    """
    rng = SplitMix64(seed)
    phases = [2.0 * math.pi * rng.uniform() for _ in range(3)]
    x = np.empty_like(X)
    for a in range(3):
        x[a] = X[a] + amp * np.sin(math.pi * X[a] + phases[a])
    return x


# ---------------------------------------------------------------- configs


@dataclass
class Workload:
    name: str
    grid: Grid
    x0: np.ndarray          # (3, nz, ny, nx) float64 initial positions x(X, 0)
    B0: np.ndarray          # (3, nz, ny, nx) float64 B(X, 0)
    steps: int              # accepted steps of the full run
    precision: str          # "fp64" | "mixed"
    curl: str               # "mimetic" | "direct"
    regions: list = field(default_factory=list)   # (xc, yc, zc, k, l, L)
    extra: dict = field(default_factory=dict)

    @property
    def theta(self):
        """Twist amplitudes then widths of the braid regions."""
        return [r[3] for r in self.regions] + [r[4] for r in self.regions]


def braid_regions(n_regions: int, seed: int | None, amp_alternating: bool,
                  l: float = 0.3, L: float = 0.25):
    rng = SplitMix64(seed) if seed is not None else None
    regs = []
    for i in range(n_regions):
        zc = -0.75 + 1.5 * i / (n_regions - 1)
        xc = 0.4 if i % 2 == 0 else -0.4
        if amp_alternating:
            k = 1.0 if i % 2 == 0 else -1.0
        else:
            k = rng.uniform_range(-1.5, 1.5)
        regs.append((xc, 0.0, zc, k, l, L))
    return regs


def braid_field(X, regions, background=(0.0, 0.0, 1.0)):
    # complex parameters give a complex field (derivatives by complex step)
    dtype = np.result_type(X, *[complex(v) if isinstance(v, complex) else float(v)
                                 for r in regions for v in r])
    B = np.zeros(X.shape, dtype=dtype)
    for c in range(3):
        B[c] += background[c]
    for (xc, yc, zc, k, l, L) in regions:
        B += twist_region(X, xc, yc, zc, k, l, L)
    return B


def braid_field_param_grad(X, regions):
    """dB0/dtheta for theta = (k_0..k_{m-1}, l_0..l_{m-1}); shape (2m, 3, ...)."""
    dk, dl = [], []
    for (xc, yc, zc, k, l, L) in regions:
        a, b = twist_region_grad(X, xc, yc, zc, k, l, L)
        dk.append(a)
        dl.append(b)
    return np.stack(dk + dl)


def make_workload(name: str, n: int | None = None, seed: int | None = None,
                  theta=None) -> Workload:
    """Build one of the named workloads; ``n`` overrides the node count per
    axis (used for small parity cases), ``theta`` overrides the braid's
    (k_i, l_i) parameters."""
    if name == "tube":
        n = n or 16
        g = Grid(n, n, n)
        X = nodes(g)
        reg = [(0.0, 0.0, 0.0, 1.0, 0.5, 1.0)]
        if theta is not None:
            reg = [(0.0, 0.0, 0.0, theta[0], theta[1], 1.0)]
        return Workload("tube", g, X.copy(), braid_field(X, reg), 200, "fp64",
                        "mimetic", reg)
    if name in ("braid", "adjoint"):
        n = n or (64 if name == "braid" else 96)
        g = Grid(n, n, n)
        X = nodes(g)
        reg = braid_regions(6, None, True)
        if theta is not None:
            m = len(reg)
            reg = [(r[0], r[1], r[2], theta[i], theta[m + i], r[5])
                   for i, r in enumerate(reg)]
        s = 2 if seed is None else seed
        steps = 2000 if name == "braid" else 500
        return Workload(name, g, predistort(X, s), braid_field(X, reg), steps,
                        "fp64", "mimetic", reg)
    if name == "braid10":
        n = n or 128
        g = Grid(n, n, n)
        X = nodes(g)
        s = 3 if seed is None else seed
        reg = braid_regions(10, s, False)
        return Workload(name, g, predistort(X, s), braid_field(X, reg), 5000,
                        "mixed", "mimetic", reg)
    if name == "prod":
        n = n or 384
        g = Grid(n, n, n)
        X = nodes(g)
        s = 5 if seed is None else seed
        reg = braid_regions(12, s, False)
        B = braid_field(X, reg) + 0.1 * abc_field(X)
        return Workload(name, g, X.copy(), B, 10000, "mixed", "mimetic", reg)
    if name == "isohelix":
        n = n or 17
        g = Grid(n, n, n, lo=(-4.0, -4.0, -10.0), hi=(4.0, 4.0, 10.0))
        X = nodes(g)
        return Workload(name, g, X.copy(), isohelix_field(X), 0, "fp64",
                        "mimetic", [])
    raise ValueError(f"unknown workload {name!r}")


WORKLOADS = {
    # name: (workload, nodes per axis, description)
    "tube16": ("tube", 16, "16^3 twisted tube, FP64 mimetic, 200 steps"),
    "braid64": ("braid", 64, "64^3 6-region braid on a pre-distorted grid, FP64, 2000 steps"),
    "braid128": ("braid10", 128, "128^3 10-region seeded braid, mixed precision, 5000 steps"),
    "adjoint96": ("adjoint", 96, "96^3 6-region braid, FP64 adjoint over 500 steps"),
    "prod384": ("prod", 384, "384^3 12-region braid + 0.1 ABC, mixed precision"),
}


# ---------------------------------------------------------------- periodic


def periodic_fields(X, P, seed=6, amp=0.05):
    """Positions and field that repeat along z with period P, sampled at the
    labels X: two twist regions modulated by sin(2 pi Z / P + phase) and
    cos(4 pi Z / P + phase) (divergence-free for any z profile) on e_z, and
    the periodic pre-distortion x_a = X_a + amp sin(pi X_a + phi_a)
    (a = x, y; the x and y faces stay planar), z = Z + amp sin(2 pi Z / P +
    phi_z).  Returns (x0, B0)."""
    rng = SplitMix64(seed)
    ph = [2.0 * math.pi * rng.uniform() for _ in range(5)]
    x, y, z = X
    w = 2.0 * math.pi / P
    G1 = np.exp(-(x * x + y * y) / 0.25) * np.sin(w * z + ph[3])
    dx2, dy2 = x - 0.3, y + 0.2
    G2 = -0.8 * np.exp(-(dx2 * dx2 + dy2 * dy2) / 0.16) * np.cos(2.0 * w * z + ph[4])
    B0 = np.stack([-y * G1 - dy2 * G2, x * G1 + dx2 * G2, np.ones_like(z)])
    x0 = np.stack([x + amp * np.sin(math.pi * x + ph[0]),
                   y + amp * np.sin(math.pi * y + ph[1]),
                   z + amp * np.sin(w * z + ph[2])])
    return x0, B0


def periodic_case(nx, ny, m, seed=6, lo_z=-1.0, h_z=2.0 / 31.0):
    """A z-periodic workload of m inner planes (period P = m h_z): the grid
    (nz = m + 2, ghost planes 0 and m+1 included) and x0, B0 of
    :func:`periodic_fields`, whose ghost nodes sit one period from their
    partners.  Returns (grid, x0, B0)."""
    g = Grid(nx, ny, m + 2, lo=(-1.0, -1.0, lo_z), hi=(1.0, 1.0, lo_z + (m + 1) * h_z),
             periodic_z=True)
    x0, B0 = periodic_fields(nodes(g), m * g.h[2], seed)
    return g, x0, B0
