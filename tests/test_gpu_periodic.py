"""Periodic z boundaries (section "Boundary Conditions": ghost planes one
period L_z + dZ from their partners; GLEMUR_FP64 two-pass stages) against
the FP64 oracle: velocities, one Cash-Karp step with both mimetic
currents, 100 steps replaying the oracle's schedule, the error control,
energy and force-free diagnostics over one period.  Tolerances as for the
line-tied path (tests/test_gpu_parity.py)."""
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


def relaxation(G, g, x0, B0, curl=0, **kw):
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, curl=curl, periodic_z=1, **kw)
    r.set_x(torch.from_numpy(np.ascontiguousarray(x0)).cuda())
    r.set_B0(torch.from_numpy(np.ascontiguousarray(B0)).cuda())
    return r


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("curl", [0, 2], ids=["mimetic", "nnn"])
@pytest.mark.parametrize("case", [(12, 10, 30), (37, 19, 21), (9, 9, 3)],
                         ids=lambda c: "x".join(map(str, c)))
def test_velocity_and_step_periodic(G, case, curl):
    g, x0, B0 = gi.periodic_case(*case)
    r = relaxation(G, g, x0, B0, curl=curl)
    u = r.velocity().cpu().numpy()
    u_ref, rc = ora.velocity(g, x0, B0, curl)
    assert rc == ora.OK
    assert rel_inf(u, u_ref) < 1e-11
    dt = 3e-4
    x_ref, lam_ref, rc = ora.step_fixed(g, x0, B0, dt, curl)
    assert rc == ora.OK
    st = r.step_fixed(dt)
    assert st["accepted"] == 1
    x = r.get_x().cpu().numpy()
    assert rel_inf(x, x_ref) < 1e-12
    assert np.abs(x - x_ref).max() < 1e-9 * np.abs(x_ref - x0).max()
    # Lambda is a cancelling sum dt sum_j (b_j - b*_j) k_j: besides 1e-9 of
    # itself it carries absolute rounding ~ eps |dt k| ~ eps |step|
    assert abs(st["lam"] - lam_ref) <= 1e-9 * lam_ref + 1e-15 * np.abs(x_ref - x0).max()
    # ghost planes: the partners' positions shifted by the period
    P = (g.nz - 2) * g.h[2]
    assert np.abs(x[2, 0] - (x[2, -2] - P)).max() < 1e-13
    assert np.abs(x[:2, -1] - x[:2, 1]).max() < 1e-14


@pytest.mark.parametrize("curl", [0, 2], ids=["mimetic", "nnn"])
def test_periodic_benchmark_size(G, curl):
    """The z-periodic 64^3 workload the benchmark times (64 x 64 nodes
    across, 62 inner planes), one step, in the benchmark's launch
    configuration (one wave of CTAs, threads taking several nodes)."""
    g, x0, B0 = gi.periodic_case(64, 64, 62, h_z=2.0 / 63.0)
    dt = 3e-4
    x_ref, lam_ref, rc = ora.step_fixed(g, x0, B0, dt, curl)
    assert rc == ora.OK
    r = relaxation(G, g, x0, B0, curl=curl)
    st = r.step_fixed(dt)
    assert st["accepted"] == 1
    x = r.get_x().cpu().numpy()
    assert rel_inf(x, x_ref) < 1e-12
    assert np.abs(x - x_ref).max() < 1e-9 * np.abs(x_ref - x0).max()
    assert abs(st["lam"] - lam_ref) <= 1e-9 * lam_ref + 1e-15 * np.abs(x_ref - x0).max()


def test_periodic_hundred_steps_replayed_and_control(G):
    g, x0, B0 = gi.periodic_case(14, 12, 20)
    x_ref, dt_ref, log, st_ref, rc = ora.relax(g, x0, B0, 100, 1e-3)
    assert rc == ora.OK and len(log) == 100
    r = relaxation(G, g, x0, B0)
    for dt in log:
        r.step_fixed(dt)
    assert rel_inf(r.get_x().cpu().numpy(), x_ref) < 1e-10
    # free-running control from the same start
    opts = ora.ControlOpts(lambda0=1e-8)
    x2, dt2, log2, st2, rc = ora.relax(g, x0, B0, 15, 5e-2, opts=opts)
    assert rc == ora.OK and st2["rejected"] > 0
    r2 = relaxation(G, g, x0, B0, lambda0=1e-8, dt0=5e-2)
    st = r2.step(15)
    assert st["accepted"] == 15 and st["rejected"] == st2["rejected"]
    assert abs(st["dt"] - dt2) < 1e-9 * dt2
    assert rel_inf(r2.get_x().cpu().numpy(), x2) < 1e-11


def test_periodic_diagnostics(G):
    g, x0, B0 = gi.periodic_case(29, 17, 24)
    r = relaxation(G, g, x0, B0)
    E_ref, _ = ora.energy(g, x0, B0)
    assert abs(r.energy() - E_ref) < 1e-13 * E_ref
    xi_ref, xis_ref, _ = ora.forcefree(g, x0, B0)
    xi, xis = r.forcefree_err()
    assert abs(xi - xi_ref) < 1e-10 * xi_ref and abs(xis - xis_ref) < 1e-10 * xis_ref
    a, e = r.alpha_line(14, 8, 1.0)
    a_o, e_o, rc = ora.alpha_line(g, x0, B0, 14, 8, 1.0)
    assert rc == ora.OK
    assert np.abs(a[1:-1] - a_o[1:-1]).max() <= 1e-10 * np.abs(a_o[1:-1]).max()
    # energy decays over the period
    E = [r.energy()]
    for _ in range(5):
        r.step(10)
        E.append(r.energy())
    assert np.all(np.diff(E) <= 1e-13 * E[0]) and E[-1] < E[0]


def test_periodic_needs_fp64_and_a_loop_current(G):
    for kw in (dict(precision=G.MIXED), dict(curl=G.DIRECT)):
        with pytest.raises(G.GlemurError):
            G.Relaxation(8, 8, 8, periodic_z=1, **kw)
