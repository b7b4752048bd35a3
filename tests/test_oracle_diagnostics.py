"""Pins of the oracle's validation diagnostics (section "Diagnostics"):
sigma_x and sigma_B, alpha* and epsilon* on a node line, and the convexity
kappa -- each against closed forms, and the IsoHelix closed-form relaxed
state against the oracle's own pull-back."""
import math

import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora


def test_deviation_closed_forms():
    """A uniform shift of every node by s gives sigma_x = |s|; a uniform
    field on x = X against B_ref = B0 + v gives sigma_B = |v| (B = B0
    exactly there)."""
    g = gi.Grid(9, 7, 8)
    X = gi.nodes(g)
    B0 = gi.uniform_field(g, (0.3, -0.2, 1.0))
    s = np.array([0.03, -0.04, 0.12])
    v = np.array([0.5, 0.0, -1.2])
    sx, sb, rc = ora.deviation(g, X + s[:, None, None, None], B0, X, B0 + v[:, None, None, None])
    assert rc == ora.OK
    assert abs(sx - np.linalg.norm(s)) < 1e-15 and abs(sb - np.linalg.norm(v)) < 1e-14


def test_isohelix_relaxed_state_is_the_pulled_back_field():
    """On the exact relaxed grid of eq. "x analytical relaxed" the pull-back
    of the IsoHelix field is B0 e_z (eq. "B relaxed") up to the Jacobian's
    discretisation error: sigma_B falls at second order with the spacing,
    and sigma_x of that grid against itself is zero."""
    errs = []
    for n in (17, 33, 65):
        w = gi.make_workload("isohelix", n=n)
        X = gi.nodes(w.grid)
        xr, Br = gi.isohelix_relaxed(X)
        sx, sb, rc = ora.deviation(w.grid, xr, w.B0, xr, Br)
        assert rc == ora.OK and sx == 0.0
        errs.append(sb)
    assert errs[0] > errs[1] > errs[2]
    # second order: the error drops ~4x per halving of h
    assert errs[1] / errs[2] > 3.5, errs


def test_alpha_of_a_linear_force_free_field():
    """B = (sin az, cos az, 1)... on x = X: curl B = a (sin az, cos az, 0)
    and the central differences of the nearest-neighbour loops (and of the
    classic current) give J = (sin(a h)/h)(sin az, cos az, 0) exactly, so
    alpha* = J.B/B^2 = (sin(a h)/h)/2 at every node of every line and
    epsilon* vanishes to rounding."""
    g = gi.Grid(7, 8, 23, (-1.0, -1.0, -2.0), (1.0, 1.0, 2.0))
    X = gi.nodes(g)
    a = 1.3
    B0 = np.stack([np.sin(a * X[2]), np.cos(a * X[2]), np.ones_like(X[2])])
    hz = g.h[2]
    for curl in (ora.MIMETIC, ora.DIRECT):
        alpha, eps, rc = ora.alpha_line(g, X, B0, 3, 4, math.sqrt(2.0), curl)
        assert rc == ora.OK
        assert np.isnan(alpha[0]) and np.isnan(alpha[-1])
        assert np.abs(alpha[1:-1] - math.sin(a * hz) / hz / 2.0).max() < 1e-13
        assert 0.0 <= eps < 1e-12


def test_epsilon_star_of_a_linear_alpha_profile():
    """B0 = (-y g(z), x g(z), 1) with g = c z / 2 on x = X (div B0 = 0): on
    the axis B = e_z and J_z = 2 g exactly (central differences of fields
    linear in x and y), so alpha* = c Z_k and every pair of axis nodes has
    slope c: epsilon* = a_r c."""
    g = gi.Grid(9, 9, 21, (-1.0, -1.0, -3.0), (1.0, 1.0, 3.0))
    X = gi.nodes(g)
    c = 0.7
    G = c * X[2] / 2.0
    B0 = np.stack([-X[1] * G, X[0] * G, np.ones_like(G)])
    a_r = 1.9
    for curl in (ora.MIMETIC, ora.DIRECT):
        alpha, eps, rc = ora.alpha_line(g, X, B0, 4, 4, a_r, curl)
        assert rc == ora.OK
        Z = X[2, 1:-1, 4, 4]
        assert np.abs(alpha[1:-1] - c * Z).max() < 1e-12
        assert abs(eps - a_r * c) < 1e-12
    # the line must be interior
    assert ora.alpha_line(g, X, B0, 0, 4, a_r)[2] == ora.ERR_BADARG


def test_convexity_closed_forms():
    """kappa = +1 everywhere on an affine grid with det A > 0 (each trihedron
    determinant is di dj dk h^3 det A), -1 everywhere on a mirrored one; a
    node pushed past its +x neighbour makes exactly that node and the
    neighbour concave (their trihedra along x flip; the others keep their
    determinant, which the x component cannot change)."""
    g = gi.Grid(6, 7, 5)
    X = gi.nodes(g)
    A = np.array([[1.1, 0.2, 0.0], [-0.1, 0.9, 0.3], [0.05, 0.0, 1.2]])
    kappa, n = ora.convexity(g, np.einsum("ab,b...->a...", A, X))
    assert n == 0 and np.all(kappa == 1)
    M = np.diag([-1.0, 1.0, 1.0])
    kappa, n = ora.convexity(g, np.einsum("ab,b...->a...", M, X))
    assert n == g.n_nodes and np.all(kappa == -1)
    x = X.copy()
    i, j, k = 2, 3, 2
    x[0, k, j, i] = X[0, k, j, i + 1] + 0.5 * g.h[0]
    kappa, n = ora.convexity(g, x)
    assert n == 2
    assert kappa[k, j, i] == -1 and kappa[k, j, i + 1] == -1
