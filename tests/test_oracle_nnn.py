"""Pins of the oracle's next-nearest-neighbour (octilateral) current,
section "Next Nearest Neighbor Mimetic Approach": exactness on affine maps,
the closed-form stencil it reduces to on a uniform grid, a brute-force
restatement of the loop integral (Gauss-Legendre edges, Newell's polygon
area) on a tiny distorted grid, second-order convergence to the analytic
current, and the one-node evaluation against the whole-grid one."""
import math

import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora
from test_oracle_pins import _analytic_case, affine_case, interior, rand_grid


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_nnn_exact_on_affine_map(seed):
    g, X, x, B0, A, G, b = affine_case(seed)
    L = A @ G @ np.linalg.inv(A) / np.linalg.det(A)
    Jex = np.array([L[2, 1] - L[1, 2], L[0, 2] - L[2, 0], L[1, 0] - L[0, 1]])
    B, _, _ = ora.pullback(g, x, B0)
    J, rc = ora.curl_nnn(g, x, B)
    assert rc == ora.OK
    assert np.abs(interior(J) - Jex[:, None, None, None]).max() <= 1e-11 * np.abs(L).max()
    Jb = J.copy()
    Jb[:, 1:-1, 1:-1, 1:-1] = 0
    assert np.all(Jb == 0)


def test_nnn_on_uniform_grid_is_the_smoothed_central_curl():
    """On x = X the octilateral is the rectangle of side 2 h_p x 2 h_q whose
    sides each take two trapezoid edges: the in-plane derivative is the
    central difference averaged across the side with weights (1/4, 1/2,
    1/4), e.g. J_z = S_y[D_x B_y] - S_x[D_y B_x]."""
    g = gi.Grid(9, 8, 10, (-1.0, -0.7, -1.2), (1.1, 0.8, 0.9))
    X = gi.nodes(g)
    rng = np.random.default_rng(4)
    B = np.stack([np.sin(1.3 * X[1] + 0.4 * X[2]) + 0.2 * X[0] ** 2,
                  np.cos(0.9 * X[2] - 0.5 * X[0]) * X[1],
                  np.sin(0.7 * X[0] * X[1]) + 0.1 * X[2]])
    B += 0.01 * rng.standard_normal(B.shape)
    J, rc = ora.curl_nnn(g, X, B)
    assert rc == ora.OK
    h = g.h

    def D(f, ax):       # central difference along label axis ax (array axis 2 - ax)
        a = 2 - ax
        return (np.roll(f, -1, a) - np.roll(f, 1, a)) / (2 * h[ax])

    def S(f, ax):       # (1/4, 1/2, 1/4) average along label axis ax
        a = 2 - ax
        return 0.25 * np.roll(f, 1, a) + 0.5 * f + 0.25 * np.roll(f, -1, a)

    Jx = S(D(B[2], 1), 2) - S(D(B[1], 2), 1)
    Jy = S(D(B[0], 2), 0) - S(D(B[2], 0), 2)
    Jz = S(D(B[1], 0), 1) - S(D(B[0], 1), 0)
    ref = np.stack([Jx, Jy, Jz])
    assert np.abs(interior(J) - interior(ref)).max() < 1e-12 * np.abs(ref).max()


def test_nnn_loop_brute_force_tiny_grid():
    """4^3 distorted grid: circulation by 3-point Gauss-Legendre quadrature
    of the linearly interpolated B along each straight edge of the eight-
    vertex loop, vector area by Newell's formula for the polygon,
    numpy.linalg.solve for J."""
    g, X, x = rand_grid(4, 5, amp=0.06)
    B0 = gi.braid_field(X, gi.braid_regions(2, None, True, l=0.7, L=0.7))
    B, _, _ = ora.pullback(g, x, B0)
    J, rc = ora.curl_nnn(g, x, B)
    assert rc == ora.OK
    gl_t = np.array([-math.sqrt(3 / 5), 0.0, math.sqrt(3 / 5)])
    gl_w = np.array([5 / 9, 8 / 9, 5 / 9])
    ring = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    for k in (1, 2):
        for j in (1, 2):
            for i in (1, 2):
                M = np.zeros((3, 3))
                circ = np.zeros(3)
                for r in range(3):
                    p, q = (r + 1) % 3, (r + 2) % 3
                    P, Bv = [], []
                    for (op, oq) in ring:
                        o = [i, j, k]
                        o[p] += op
                        o[q] += oq
                        P.append(x[:, o[2], o[1], o[0]])
                        Bv.append(B[:, o[2], o[1], o[0]])
                    s = 0.0
                    for m in range(8):
                        a0, a1 = P[m], P[(m + 1) % 8]
                        b0, b1 = Bv[m], Bv[(m + 1) % 8]
                        for t, wgt in zip(gl_t, gl_w):
                            lam = 0.5 * (t + 1)
                            s += 0.5 * wgt * np.dot((1 - lam) * b0 + lam * b1, a1 - a0)
                    circ[r] = s
                    M[r] = 0.5 * sum(np.cross(P[m], P[(m + 1) % 8]) for m in range(8))
                Jb = np.linalg.solve(M, circ)
                assert np.abs(Jb - J[:, k, j, i]).max() < 1e-12 * max(1.0, np.abs(Jb).max())


def test_nnn_converges_second_order_on_nonlinear_map():
    f = _analytic_case()
    errs = []
    for n in (9, 17, 33):
        g = gi.Grid(n, n, n, (-0.6,) * 3, (0.6,) * 3)
        X = gi.nodes(g)
        xs, B0s, Bs, Js = f(X[0], X[1], X[2])
        x = np.stack([np.broadcast_to(v, X[0].shape) for v in xs]).astype(np.float64)
        B0 = np.stack([np.broadcast_to(v, X[0].shape) for v in B0s]).astype(np.float64)
        Jex = np.stack([np.broadcast_to(v, X[0].shape) for v in Js]).astype(np.float64)
        B, _, _ = ora.pullback(g, x, B0)
        J, rc = ora.curl_nnn(g, x, B)
        assert rc == ora.OK
        errs.append(np.abs(interior(J) - interior(Jex)).max())
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.5, errs


def test_nnn_velocity_at_matches_the_field():
    g, X, x = rand_grid(7, 8, amp=0.04)
    B0 = gi.braid_field(X, gi.braid_regions(3, 2, False, l=0.6, L=0.6))
    u, rc = ora.velocity(g, x, B0, ora.NNN)
    assert rc == ora.OK
    for (i, j, k) in [(1, 1, 1), (3, 4, 2), (5, 5, 5), (0, 3, 3)]:
        un, rc = ora.velocity_at(g, x, B0, i, j, k, ora.NNN)
        assert rc == ora.OK
        assert np.abs(un - u[:, k, j, i]).max() <= 1e-14 * max(1.0, np.abs(u).max())


def test_octilateral_area_and_circulation_depend_on_the_loop_only():
    """The form the GPU pass evaluates: for any eight vertices (not planar),
    the paper's area decomposition -- the four corner triangles (edges
    meeting at V_2k+1 .. V_2k+3, / 2) plus the inner quadrilateral through
    V_2, V_4, V_6, V_8 (/ 4) -- is the vector area of the closed loop,
    1/2 sum_m r_m x r_m+1, whatever the origin; and the edge-mean
    circulation sum_m (B_m + B_m+1)/2 . (r_m+1 - r_m) equals
    sum_m B_m . (r_m+1 - r_m-1) / 2.  A dropped triangle, a wrong weight on
    the quadrilateral or a shifted B index fails it."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        r = rng.normal(size=(8, 3)) + rng.normal(size=3)
        B = rng.normal(size=(8, 3))
        dx = np.roll(r, -1, axis=0) - r                      # dx_m = r_m+1 - r_m
        corners = sum(np.cross(dx[2 * t + 1], dx[(2 * t + 2) % 8]) for t in range(4)) / 2
        quad = r[[3, 5, 7, 1]] - r[[1, 3, 5, 7]]             # V2->V4->V6->V8->V2
        inner = sum(np.cross(quad[t], quad[(t + 1) % 4]) for t in range(4)) / 4
        loop = sum(np.cross(r[m], r[(m + 1) % 8]) for m in range(8)) / 2
        assert np.allclose(corners + inner, loop, rtol=0, atol=1e-12 * np.abs(r).max() ** 2)
        shifted = r - rng.normal(size=3)
        loop2 = sum(np.cross(shifted[m], shifted[(m + 1) % 8]) for m in range(8)) / 2
        assert np.allclose(loop2, loop, rtol=0, atol=1e-11 * np.abs(r).max() ** 2)
        edge = sum((B[m] + B[(m + 1) % 8]) @ dx[m] for m in range(8)) / 2
        vert = sum(B[m] @ (r[(m + 1) % 8] - r[m - 1]) for m in range(8)) / 2
        assert abs(edge - vert) <= 1e-12 * np.abs(B).max() * np.abs(r).max()
