"""Pins of the oracle's periodic z boundary (section "Boundary Conditions":
ghost planes one period L_z + dZ from their partners): a periodic step
equals a line-tied step on a grid three periods long at the nodes of its
middle period (whose dependency cones stay clear of the line-tied ends);
shifting the state by whole planes commutes with stepping; the ghost
planes stay shifted copies; the energy of a uniform field is exactly one
period's."""
import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora


def test_periodic_step_equals_the_middle_of_a_tiled_line_tied_grid():
    m = 30
    g, x0, B0 = gi.periodic_case(12, 10, m)
    h = g.h
    P = m * h[2]
    # three periods plus two end planes, line-tied, same labels shifted
    gt = gi.Grid(g.nx, g.ny, 3 * m + 2, lo=(g.lo[0], g.lo[1], g.lo[2] - m * h[2]),
                 hi=(g.hi[0], g.hi[1], g.lo[2] + (2 * m + 1) * h[2]))
    assert abs(gt.h[2] - h[2]) < 1e-15
    xt, Bt = gi.periodic_fields(gi.nodes(gt), P)
    dt = 3e-4
    xp, lam_p, rc = ora.step_fixed(g, x0, B0, dt)
    assert rc == ora.OK
    xtn, _, rc = ora.step_fixed(gt, xt, Bt, dt)
    assert rc == ora.OK
    # periodic inner plane k <-> tiled plane k + m (labels coincide)
    mid = xtn[:, m + 1:2 * m + 1]
    inner = xp[:, 1:m + 1]
    step = np.abs(inner - x0[:, 1:m + 1]).max()
    assert step > 1e-5
    assert np.abs(mid - inner).max() < 1e-12 * step + 1e-14


def test_shifting_by_whole_planes_commutes_with_stepping():
    m = 24
    g, x0, B0 = gi.periodic_case(11, 9, m)
    s = 7
    P = m * g.h[2]
    ez = np.array([0.0, 0.0, 1.0])[:, None, None, None]

    def shift(v, with_positions):
        """Inner plane k takes plane k - s (mod m); positions move by s h_z."""
        out = v.copy()
        inner = v[:, 1:m + 1]
        rolled = np.roll(inner, s, axis=1)
        if with_positions:
            # planes that wrapped around came from one period higher
            rolled = rolled + s * g.h[2] * ez
            rolled[:, :s] -= P * ez
        out[:, 1:m + 1] = rolled
        return out

    x_s = shift(x0, True)
    B_s = shift(B0, False)
    # ghost planes follow from the inner ones
    x_s[:, 0] = x_s[:, m] - P * ez[:, 0]
    x_s[:, m + 1] = x_s[:, 1] + P * ez[:, 0]
    B_s[:, 0], B_s[:, m + 1] = B_s[:, m], B_s[:, 1]
    dt = 4e-4
    a = x0.copy()
    b = x_s.copy()
    for _ in range(3):
        a, _, rc = ora.step_fixed(g, a, B0, dt)
        assert rc == ora.OK
        b, _, rc = ora.step_fixed(g, b, B_s, dt)
        assert rc == ora.OK
    a_s = shift(a, True)
    assert np.abs(a_s[:, 1:m + 1] - b[:, 1:m + 1]).max() < 1e-13
    # ghost planes stay shifted copies of their partners
    assert np.array_equal(b[:, 0], b[:, m] - P * ez[:, 0])
    assert np.array_equal(b[:, m + 1], b[:, 1] + P * ez[:, 0])


def test_periodic_energy_of_a_uniform_field_is_one_period():
    g, _, _ = gi.periodic_case(9, 8, 12)
    X = gi.nodes(g)
    E, rc = ora.energy(g, X, gi.uniform_field(g, (0.0, 0.0, 1.5)))
    assert rc == ora.OK
    vol = (g.hi[0] - g.lo[0]) * (g.hi[1] - g.lo[1]) * 12 * g.h[2]
    assert abs(E - 0.5 * 1.5 ** 2 * vol) < 1e-14 * E


def test_periodic_single_node_velocity_is_refused():
    g, x0, B0 = gi.periodic_case(6, 6, 6)
    assert ora.velocity_at(g, x0, B0, 2, 2, 2)[1] == ora.ERR_BADARG
