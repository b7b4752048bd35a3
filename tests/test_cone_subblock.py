"""The dependency-cone sub-block (tests/cone.py) reproduces whole-grid
oracle steps exactly: the property the full-size sampled parity tests rest
on, checked on grids the oracle steps whole."""
import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora
from cone import RADIUS, subblock


@pytest.mark.parametrize("curl", [ora.MIMETIC, ora.DIRECT], ids=["mimetic", "direct"])
def test_subblock_step_equals_whole_grid_step(curl):
    g = gi.Grid(40, 34, 37)
    X = gi.nodes(g)
    x0 = gi.predistort(X, 2)
    B0 = gi.braid_field(X, gi.braid_regions(6, None, True))
    dt = 3e-4
    x_ref, _, rc = ora.step_fixed(g, x0, B0, dt, curl)
    assert rc == ora.OK
    # interior node far from every face, nodes near faces and a corner
    for (i, j, k) in [(20, 17, 18), (1, 1, 1), (38, 32, 35), (3, 30, 18), (20, 2, 34)]:
        sub, xs, bs, (a, b, c) = subblock(g, x0, B0, i, j, k)
        xn, _, rc = ora.step_fixed(sub, xs, bs, dt, curl)
        assert rc == ora.OK
        assert np.array_equal(xn[:, c, b, a], x_ref[:, k, j, i]), (i, j, k)


def test_subblock_radius_is_needed():
    """A sub-block too small for the cone does change the result (so the
    test above is not vacuous): with half-width 8 the centre moves."""
    g = gi.Grid(40, 34, 37)
    X = gi.nodes(g)
    x0 = gi.predistort(X, 2)
    B0 = gi.braid_field(X, gi.braid_regions(6, None, True))
    dt = 3e-4
    x_ref, _, _ = ora.step_fixed(g, x0, B0, dt)
    sub, xs, bs, (a, b, c) = subblock(g, x0, B0, 20, 17, 18, radius=8)
    xn, _, _ = ora.step_fixed(sub, xs, bs, dt)
    assert not np.array_equal(xn[:, c, b, a], x_ref[:, 18, 17, 20])
    assert RADIUS >= 13
