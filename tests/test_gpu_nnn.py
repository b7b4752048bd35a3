"""The next-nearest-neighbour (octilateral) current of section "Next
Nearest Neighbor Mimetic Approach" (GLEMUR_CURL_NNN, FP64 two-pass stages)
against the FP64 oracle: velocities, one Cash-Karp step (also at the 64^3
benchmark size, where threads take several nodes), the force-free
diagnostics and alpha* along a node line.  Tolerances as for the
nearest-neighbour current (tests/test_gpu_parity.py)."""
import math

import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_0942_gb300 as pkg
    pkg.lib()
    return pkg


def braid_case(nx, ny, nz):
    g = gi.Grid(nx, ny, nz)
    X = gi.nodes(g)
    return g, gi.predistort(X, 2), gi.braid_field(X, gi.braid_regions(6, None, True))


def relaxation(G, g, x0, B0, **kw):
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, curl=G.NNN, **kw)
    r.set_x(torch.from_numpy(np.ascontiguousarray(x0)).cuda())
    r.set_B0(torch.from_numpy(np.ascontiguousarray(B0)).cuda())
    return r


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("dims", [(3, 3, 3), (16, 16, 16), (37, 19, 23)],
                         ids=lambda d: "x".join(map(str, d)))
def test_velocity_nnn(G, dims):
    g, x0, B0 = braid_case(*dims)
    r = relaxation(G, g, x0, B0)
    u = r.velocity().cpu().numpy()
    u_ref, rc = ora.velocity(g, x0, B0, ora.NNN)
    assert rc == ora.OK
    assert rel_inf(u, u_ref) < 1e-11
    ub = u.copy()
    ub[:, 1:-1, 1:-1, 1:-1] = 0
    assert np.all(ub == 0)


@pytest.mark.parametrize("dims", [(24, 20, 28), (64, 64, 64)], ids=lambda d: "x".join(map(str, d)))
def test_one_step_nnn(G, dims):
    g, x0, B0 = braid_case(*dims)
    dt = 3e-4
    x_ref, lam_ref, rc = ora.step_fixed(g, x0, B0, dt, ora.NNN)
    assert rc == ora.OK
    r = relaxation(G, g, x0, B0)
    st = r.step_fixed(dt)
    assert st["accepted"] == 1
    x = r.get_x().cpu().numpy()
    assert rel_inf(x, x_ref) < 1e-12
    assert np.abs(x - x_ref).max() < 1e-9 * np.abs(x_ref - x0).max()
    # Lambda is a cancelling sum dt sum_j (b_j - b*_j) k_j: besides 1e-9 of
    # itself it carries absolute rounding ~ eps |dt k| ~ eps |step|
    assert abs(st["lam"] - lam_ref) <= 1e-9 * lam_ref + 1e-15 * np.abs(x_ref - x0).max()


def test_diagnostics_nnn(G):
    g, x0, B0 = braid_case(29, 17, 21)
    r = relaxation(G, g, x0, B0)
    xi_ref, xis_ref, _ = ora.forcefree(g, x0, B0, ora.NNN)
    xi, xis = r.forcefree_err()
    assert abs(xi - xi_ref) < 1e-10 * xi_ref and abs(xis - xis_ref) < 1e-10 * xis_ref
    E_ref, _ = ora.energy(g, x0, B0)
    assert abs(r.energy() - E_ref) < 1e-13 * E_ref
    a, e = r.alpha_line(14, 8, math.sqrt(2.0))
    a_o, e_o, rc = ora.alpha_line(g, x0, B0, 14, 8, math.sqrt(2.0), ora.NNN)
    assert np.abs(a[1:-1] - a_o[1:-1]).max() <= 1e-10 * np.abs(a_o[1:-1]).max()
    assert abs(e - e_o) <= 1e-8 * e_o


def test_nnn_is_fp64_only(G):
    with pytest.raises(G.GlemurError):
        G.Relaxation(8, 8, 8, precision=G.MIXED, curl=G.NNN)


def _isohelix(G, n, phi, curl, mult):
    w = gi.make_workload("isohelix", n=n)
    g = w.grid
    X = gi.nodes(g)
    B0 = gi.isohelix_field(X, phi=phi)
    xr, Br = gi.isohelix_relaxed(X, phi=phi)
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, curl=curl, dt0=1e-2, safety=0.9)
    r.set_x(torch.from_numpy(np.ascontiguousarray(w.x0)).cuda())
    r.set_B0(torch.from_numpy(np.ascontiguousarray(B0)).cuda())
    try:
        r.step(mult * 1200 * (n - 1) ** 2 // 256)
    except G.GlemurError as e:
        return e.code
    c = (n - 1) // 2
    _, eps = r.alpha_line(c, c, math.sqrt(2.0))
    sx, sb = r.deviation(torch.from_numpy(xr).cuda(), torch.from_numpy(Br).cuda())
    return {"eps_star": eps, "sigma_B": sb, "sigma_x": sx, "xi": r.forcefree_err()[0]}


def test_nnn_isohelix_against_the_papers_findings(G):
    """The paper's findings for the next-nearest-neighbour current
    (section "Next-Nearest-Neighbors Mimetic Approach", IsoHelix): at
    phi = pi/4, sigma_x and xi behave almost as with the nearest-neighbour
    current while epsilon* improves by up to five orders of magnitude --
    here sigma_x within 2 %, sigma_B within 35 %, and epsilon* 5e3 (n = 17)
    and 3e5 (n = 33) times smaller; and the method is unstable for the
    stronger twists -- here at phi = pi (n = 33) its step size collapses
    while the nearest-neighbour run completes.  (At phi = pi/2 this
    library's octilateral current, reading of the missing figure, stays
    stable over the run, unlike the paper's.)"""
    for n, ratio in ((17, 1e3), (33, 1e5)):
        m = _isohelix(G, n, math.pi / 4, G.MIMETIC, 4)
        q = _isohelix(G, n, math.pi / 4, G.NNN, 4)
        assert isinstance(m, dict) and isinstance(q, dict), (m, q)
        assert q["sigma_x"] == pytest.approx(m["sigma_x"], rel=0.02)
        assert q["sigma_B"] == pytest.approx(m["sigma_B"], rel=0.35)
        assert q["xi"] < 10 * max(m["xi"], 1e-6)
        assert q["eps_star"] * ratio < m["eps_star"], (n, q["eps_star"], m["eps_star"])
    assert isinstance(_isohelix(G, 33, math.pi, G.MIMETIC, 1), dict)
    assert _isohelix(G, 33, math.pi, G.NNN, 1) == -5       # GLEMUR_ERR_DT_UNDERFLOW
