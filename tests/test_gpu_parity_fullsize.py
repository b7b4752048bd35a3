"""Full Cash-Karp steps at the benchmark sizes, in the launch configurations
the benchmark times, against the FP64 oracle.

* FP64 two-pass stages on the 64^3 braid (the benchmark's workload; each
  pass runs one wave of CTAs, so some threads take two nodes) and on the
  96^3 braid (every thread takes at least five interior nodes in every
  pass, so the grid-stride loops of both passes run several times);
* the direct current on the 64^3 braid (FP64 and mixed precision);
* mixed precision on the 128^3 ten-region braid: TMA tiles (19 z-planes per
  CTA, the multi-plane ring) and the register-staged tiles;
* five error-controlled steps on the 64^3 braid (accept/reject sequence,
  step sizes, positions);
* the 384^3 production workload (mixed precision), one step, checked at
  sampled nodes against oracle steps on sub-blocks that hold each node's
  whole dependency cone (tests/cone.py; the CPU test
  tests/test_cone_subblock.py checks that such a sub-block reproduces a
  whole-grid oracle step bit for bit).

Tolerances are those of tests/test_gpu_parity.py: FP64 x within 1e-12
relative per step and the step's displacement within 1e-9 of its size, the
error norm within 1e-9; mixed precision the step's displacement within
3e-4 of its size plus FP32 rounding of the stored displacement.
"""
import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora
from cone import subblock

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_0942_gb300 as pkg
    pkg.lib()
    return pkg


_W = {}


def workload(name):
    if name not in _W:
        base, n, _ = gi.WORKLOADS[name]
        _W[name] = gi.make_workload(base, n=n)
    return _W[name]


def relaxation(G, w, precision=0, curl=0, **kw):
    g = w.grid
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, precision=precision, curl=curl, **kw)
    r.set_x(torch.from_numpy(w.x0).cuda())
    r.set_B0(torch.from_numpy(w.B0).cuda())
    return r


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def check_fp64_step(G, w, dt, curl):
    x_ref, lam_ref, rc = ora.step_fixed(w.grid, w.x0, w.B0, dt, curl)
    assert rc == ora.OK
    r = relaxation(G, w, curl=curl)
    st = r.step_fixed(dt)
    assert st["accepted"] == 1 and st["status"] == 0
    x = r.get_x().cpu().numpy()
    assert rel_inf(x, x_ref) < 1e-12
    step = np.abs(x_ref - w.x0).max()
    assert np.abs(x - x_ref).max() < 1e-9 * step
    # Lambda: 1e-9 of itself plus absolute rounding ~ eps |step| (a
    # cancelling sum of the stage derivatives)
    assert abs(st["lam"] - lam_ref) <= 1e-9 * lam_ref + 1e-15 * step
    return r, x_ref


def check_mixed_step(G, w, dt, curl):
    X = gi.nodes(w.grid)
    x_ref, lam_ref, rc = ora.step_fixed(w.grid, w.x0, w.B0, dt, curl)
    assert rc == ora.OK
    r = relaxation(G, w, precision=1, curl=curl)
    st = r.step_fixed(dt)
    assert st["accepted"] == 1 and st["status"] == 0
    x = r.get_x().cpu().numpy()
    step = np.abs(x_ref - w.x0).max()
    err = np.abs(x - x_ref).max()
    assert err <= 3e-4 * step + 2e-7 * np.abs(x_ref - X).max(), (err, step)
    assert abs(st["lam"] - lam_ref) <= 5e-2 * lam_ref, (st["lam"], lam_ref)
    return r, x_ref


def test_full_step_fp64_braid64(G):
    w = workload("braid64")
    r, x_ref = check_fp64_step(G, w, 3e-4, 0)
    E_ref, _ = ora.energy(w.grid, x_ref, w.B0)
    assert abs(r.energy() - E_ref) <= 1e-13 * E_ref


def test_full_step_fp64_adjoint96_multi_node_threads(G):
    w = workload("adjoint96")
    # the two-pass grids hold at most 4 CTAs of 256 threads per SM
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert w.grid.n_interior >= 5 * 4 * 256 * nsm
    check_fp64_step(G, w, 3e-4, 0)


def test_full_step_fp64_direct_braid64(G):
    check_fp64_step(G, workload("braid64"), 3e-4, 1)


def test_full_step_mixed_direct_braid64(G):
    check_mixed_step(G, workload("braid64"), 3e-4, 1)


@pytest.mark.parametrize("tma", ["1", "0"], ids=["tma", "registers"])
def test_full_step_mixed_braid128(G, tma, monkeypatch):
    monkeypatch.setenv("GLEMUR_TMA", tma)
    w = workload("braid128")
    r, x_ref = check_mixed_step(G, w, 1e-4, 0)
    E_ref, _ = ora.energy(w.grid, x_ref, w.B0)
    assert abs(r.energy() - E_ref) <= 1e-6 * E_ref
    del r
    torch.cuda.empty_cache()


def test_controlled_steps_fp64_braid64(G):
    """Five error-controlled steps from dt0 = 1e-3 (the first attempts are
    rejected): the same accept/reject sequence, step size and time as the
    oracle's control, positions within 1e-11 relative."""
    w = workload("braid64")
    x_ref, dt_ref, log, st_ref, rc = ora.relax(w.grid, w.x0, w.B0, 5, 1e-3)
    assert rc == ora.OK and st_ref["rejected"] > 0
    r = relaxation(G, w, dt0=1e-3)
    st = r.step(5)
    assert st["accepted"] == 5 and st["rejected"] == st_ref["rejected"]
    assert abs(st["dt"] - dt_ref) < 1e-9 * dt_ref
    assert abs(st["t"] - st_ref["t"]) < 1e-9 * st_ref["t"]
    assert abs(st["dt_last"] - log[-1]) < 1e-9 * log[-1]
    # the device-side log of accepted step sizes is the oracle's schedule
    sched = r.dt_schedule(0, 5)
    assert np.abs(sched - log).max() < 1e-9 * log.max()
    with pytest.raises(G.GlemurError):
        r.dt_schedule(3, 3)                  # step 5 has not been taken
    assert rel_inf(r.get_x().cpu().numpy(), x_ref) < 1e-11


def _sample_nodes(g, count, seed):
    rng = np.random.default_rng(seed)
    pts = [(1, 1, 1), (g.nx - 2, g.ny - 2, g.nz - 2), (g.nx // 2, g.ny // 2, g.nz // 2),
           (1, g.ny - 2, g.nz // 3), (g.nx - 2, 1, 2)]
    for _ in range(count):
        pts.append(tuple(int(rng.integers(1, n - 1)) for n in (g.nx, g.ny, g.nz)))
    return pts


def test_full_step_prod384_sampled_mixed(G):
    """The 384^3 production workload, one mixed-precision step in the
    benchmark's launch configuration; at sampled nodes the updated
    positions against oracle steps on dependency-cone sub-blocks."""
    w = workload("prod384")
    g = w.grid
    dt = 1e-5   # h = 2/383: larger steps fold trial stages (1e-4 does)
    r = relaxation(G, w, precision=1)
    st = r.step_fixed(dt)
    assert st["accepted"] == 1 and st["status"] == 0
    x = r.get_x()
    for (i, j, k) in _sample_nodes(g, 12, 3):
        sub, xs, bs, (a, b, c) = subblock(g, w.x0, w.B0, i, j, k)
        xn, _, rc = ora.step_fixed(sub, xs, bs, dt)
        assert rc == ora.OK
        scale = np.abs(xn - xs).max()
        got = x[:, k, j, i].cpu().numpy()
        want = xn[:, c, b, a]
        # x0 = X here, so want - x0 is the displacement the FP32 state stores
        tol = 3e-4 * scale + 2e-7 * np.abs(want - xs[:, c, b, a]).max()
        assert np.abs(got - want).max() <= tol, (i, j, k, got, want, scale)
    del r, x
    _W.pop("prod384")
    torch.cuda.empty_cache()


def test_braid64_two_thousand_steps_mimetic_and_direct(G):
    """The 64^3 braid configuration as specified: 2000 error-controlled FP64
    steps with each current (step-size safety 0.9).  Both runs finish with
    the energy falling at every 100 steps; the force-free error xi falls in
    both, and further with the mimetic current than with the direct one
    (the paper's comparison of the two)."""
    w = workload("braid64")
    out = {}
    for curl in (0, 1):
        r = relaxation(G, w, curl=curl, safety=0.9)
        E = [r.energy()]
        xi0 = r.forcefree_err()[0]
        for c in range(20):
            st = r.step(100)
            assert st["status"] == 0 and st["accepted"] == 100 * (c + 1)   # cumulative
            E.append(r.energy())
        E = np.array(E)
        assert np.all(np.diff(E) <= 1e-13 * E[0]) and E[-1] < E[0]
        xi = r.forcefree_err()[0]
        assert xi < xi0
        out[curl] = (E[-1], xi, r.stats()["t"])
    print("2000 steps (E_M, xi, t):", out)
    assert out[0][1] < out[1][1], out
