"""The oracle against the numbers the paper prints for its IsoHelix
experiment (Table 1, phi = pi/4, double precision; fixture
tests/golden/isohelix_table1.json): relax the IsoHelix field (eq. "B init
analytical", box 8 x 8 x 20, 17^3 nodes) to its asymptotic state and take
epsilon* on the central line (eq. "epsilon star"), sigma_B and sigma_x
against the closed-form relaxed state (eqs. "B relaxed", "x analytical
relaxed").

The nearest-neighbour mimetic run reproduces the printed values to within
a few per cent (the paper gives neither Lambda_0 nor the run length; the
values have settled by 600 steps here).  The classic current is this
library's reading of a formula the paper does not print (its parity is
unpinned): the test holds it only to the paper's qualitative statement --
epsilon* of order one, more than ten times the mimetic value -- and to the
printed sigma_B within a factor of two.
"""
import functools
import json
import math
import os

import pytest

import glemur_inputs as gi
import oracle as ora

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = json.load(open(os.path.join(HERE, "golden", "isohelix_table1.json")))


@functools.lru_cache(maxsize=None)
def relaxed_diagnostics(n, curl, steps):
    w = gi.make_workload("isohelix", n=n)
    g = w.grid
    xr, Br = gi.isohelix_relaxed(gi.nodes(g), phi=TABLE["phi"])
    opts = ora.ControlOpts(safety=0.9)
    x, _, _, st, rc = ora.relax(g, w.x0, w.B0, steps, 1e-2, curl, opts=opts)
    assert rc == ora.OK
    c = (n - 1) // 2
    _, eps, rc = ora.alpha_line(g, x, w.B0, c, c, math.sqrt(2.0), curl)
    assert rc == ora.OK
    sx, sb, _ = ora.deviation(g, x, w.B0, xr, Br)
    return eps, sb, sx


def test_mimetic_reproduces_table1_n17():
    eps, sb, sx = relaxed_diagnostics(17, ora.MIMETIC, 600)
    ref = TABLE["mimetic"]["17"]
    assert eps == pytest.approx(ref["eps_star"], rel=0.1)
    assert sb == pytest.approx(ref["sigma_B"], rel=0.1)
    assert sx == pytest.approx(ref["sigma_x"], rel=0.1)


def test_classic_is_qualitatively_table1_n17():
    eps_m, sb_m, _ = relaxed_diagnostics(17, ora.MIMETIC, 600)
    eps_c, sb_c, _ = relaxed_diagnostics(17, ora.DIRECT, 600)
    ref = TABLE["classic"]["17"]
    assert 0.1 < eps_c < 2.0 and eps_c > 10 * eps_m
    assert 0.5 * ref["sigma_B"] < sb_c < 2.0 * ref["sigma_B"]
    assert sb_c > 5 * sb_m


def test_mimetic_reproduces_table1_pi_over_2_n17():
    """Table 1's phi = pi/2 row (single precision in the paper; fixture
    tests/golden/isohelix_table1_single.json) at n = 17: epsilon*, sigma_B
    and sigma_x are set by the discretisation, so the FP64 oracle's run
    reproduces them (within 6 % after 600 steps)."""
    ref = json.load(open(os.path.join(HERE, "golden", "isohelix_table1_single.json")))
    ref = ref["mimetic"]["pi/2"]["17"]
    w = gi.make_workload("isohelix", n=17)
    g = w.grid
    X = gi.nodes(g)
    B0 = gi.isohelix_field(X, phi=math.pi / 2)
    xr, Br = gi.isohelix_relaxed(X, phi=math.pi / 2)
    x, _, _, st, rc = ora.relax(g, w.x0, B0, 600, 1e-2, ora.MIMETIC,
                                opts=ora.ControlOpts(safety=0.9))
    assert rc == ora.OK
    _, eps, rc = ora.alpha_line(g, x, B0, 8, 8, math.sqrt(2.0), ora.MIMETIC)
    assert rc == ora.OK
    sx, sb, _ = ora.deviation(g, x, B0, xr, Br)
    assert eps == pytest.approx(ref["eps_star"], rel=0.1)
    assert sb == pytest.approx(ref["sigma_B"], rel=0.1)
    assert sx == pytest.approx(ref["sigma_x"], rel=0.1)


def test_pontin09_reproduces_table2_n17():
    """Table 2's mimetic row at n = 17 (Pontin09, twists +-pi/2; fixture
    tests/golden/pontin09_table2.json), the oracle with the offset reading
    +-4 (glemur_inputs.PONTIN09_L): epsilon* within 10 % after 600 steps
    (0.118 against 0.11)."""
    ref = json.load(open(os.path.join(HERE, "golden", "pontin09_table2.json")))
    w = gi.make_workload("isohelix", n=17)
    g = w.grid
    B0 = gi.pontin09_field(gi.nodes(g))
    x, _, _, st, rc = ora.relax(g, w.x0, B0, 600, 1e-2, ora.MIMETIC,
                                opts=ora.ControlOpts(safety=0.9))
    assert rc == ora.OK
    _, eps, rc = ora.alpha_line(g, x, B0, 8, 8, math.sqrt(2.0), ora.MIMETIC)
    assert rc == ora.OK
    assert eps == pytest.approx(ref["mimetic"]["17"]["eps_star"], rel=0.1)
