"""The seeded input generators (glemur_inputs): every initial field the
workloads use is solenoidal (its divergence, by fourth-order differences on
a fine grid, vanishes to the differences' truncation), the IsoHelix and
Pontin09 fields follow their equations at sample points, Pontin09 with
opposite twists at +-L is odd under Z -> -Z in its transverse part, and the
IsoHelix relaxed state leaves the far field in place."""
import math

import numpy as np
import pytest

import glemur_inputs as gi


def _div4(B, h):
    """Fourth-order central divergence at the points two away from every face."""
    def d(f, ax, hh):
        s = [slice(2, -2)] * 3
        def sh(k):
            t = list(s)
            t[ax] = slice(2 + k, f.shape[ax] - 2 + k)
            return f[tuple(t)]
        return (-sh(2) + 8 * sh(1) - 8 * sh(-1) + sh(-2)) / (12 * hh)
    # B[c] has axes (z, y, x): component x varies along axis 2, y along 1, z along 0
    return d(B[0], 2, h[0]) + d(B[1], 1, h[1]) + d(B[2], 0, h[2])


@pytest.mark.parametrize("name", ["braid", "abc", "isohelix", "pontin09", "periodic"])
def test_fields_are_solenoidal(name):
    if name in ("isohelix", "pontin09"):
        g = gi.Grid(41, 41, 81, lo=(-4.0, -4.0, -10.0), hi=(4.0, 4.0, 10.0))
    else:
        g = gi.Grid(49, 47, 45)
    X = gi.nodes(g)
    if name == "braid":
        B = gi.braid_field(X, gi.braid_regions(6, None, True))
    elif name == "abc":
        B = gi.abc_field(X)
    elif name == "isohelix":
        B = gi.isohelix_field(X, phi=math.pi / 2)
    elif name == "pontin09":
        B = gi.pontin09_field(X)
    else:
        _, B = gi.periodic_fields(X, 2.0, seed=6)
    h = np.array(g.h)
    div = _div4(B, h)
    scale = max(np.abs(np.diff(B[c], axis=a)).max() / h[2 - a]
                for c in range(3) for a in range(3))
    assert np.abs(div).max() < 2e-3 * scale, (name, np.abs(div).max(), scale)


def test_isohelix_and_pontin09_follow_their_equations():
    rng = np.random.default_rng(5)
    P = np.stack([rng.uniform(-4, 4, 7), rng.uniform(-4, 4, 7), rng.uniform(-10, 10, 7)])
    X = P[:, :, None, None]
    a_r, a_z, phi = math.sqrt(2.0), 2.0, 0.7
    B = gi.isohelix_field(X, phi=phi)[:, :, 0, 0]
    for m in range(7):
        x, y, z = P[:, m]
        f = 2.0 * z / a_z ** 2 * math.exp(-(x * x + y * y) / a_r ** 2 - z * z / a_z ** 2) * phi
        assert B[:, m] == pytest.approx([f * y, -f * x, 1.0], rel=1e-14, abs=1e-15)
    B = gi.pontin09_field(X, phi=(0.9, -0.4), L=(3.0, -2.5))[:, :, 0, 0]
    for m in range(7):
        x, y, z = P[:, m]
        e = sum(2.0 * ph / (math.pi * a_r) * math.exp(-(x * x + y * y) / a_r ** 2
                                                      - (z - L) ** 2 / a_z ** 2)
                for ph, L in ((0.9, 3.0), (-0.4, -2.5)))
        assert B[:, m] == pytest.approx([-y * e, x * e, 1.0], rel=1e-14, abs=1e-15)


def test_pontin09_opposite_twists_are_odd_in_z():
    g = gi.Grid(17, 17, 33, lo=(-4.0, -4.0, -10.0), hi=(4.0, 4.0, 10.0))
    X = gi.nodes(g)
    B = gi.pontin09_field(X)
    # node k and nz-1-k mirror each other in Z
    assert np.allclose(B[:2], -B[:2, ::-1], rtol=0, atol=1e-15)
    assert np.all(B[2] == 1.0)


def test_isohelix_relaxed_state_keeps_the_far_field():
    g = gi.Grid(17, 17, 33, lo=(-4.0, -4.0, -10.0), hi=(4.0, 4.0, 10.0))
    X = gi.nodes(g)
    xr, Br = gi.isohelix_relaxed(X, phi=math.pi)
    far = np.exp(-(X[0] ** 2 + X[1] ** 2) / 2.0 - X[2] ** 2 / 4.0) < 1e-12
    assert np.allclose(xr[:, far], X[:, far], rtol=0, atol=1e-10)   # turn < pi 1e-12, r < 6
    assert np.all(xr[2] == X[2]) and np.all(Br[2] == 1.0) and np.all(Br[:2] == 0.0)
    # the axis does not move, and the turn keeps each node's distance from it
    r0 = np.hypot(X[0], X[1])
    assert np.allclose(np.hypot(xr[0], xr[1]), r0, rtol=0, atol=1e-12)
