"""The 384^3 production workload as configured (12 seeded twist regions plus
0.1 ABC on e_z, about 57M nodes): 10000 error-controlled mixed-precision
steps (FP32 fields, FP64 reductions and control, step-size safety 0.9),
then the mixed-precision adjoint over the last 200 of them.  The energy
must fall monotonically over the run and xi fall; the adjoint's loss and
its parameter gradient (amplitudes and widths of three regions) must agree
with an FP64 context's adjoint over the same 200 steps (the same start
state and step sizes) to 1e-6 relative -- on a GB300 they
agree to about 1e-8.  About four minutes and 125 GB of device memory."""
import numpy as np
import pytest

import glemur_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_0942_gb300 as pkg
    pkg.lib()
    return pkg


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_prod384_ten_thousand_steps_and_mixed_adjoint(G):
    free, _ = torch.cuda.mem_get_info()
    if free < 140e9:
        pytest.skip("needs about 140 GB of free device memory")
    base, n, _ = gi.WORKLOADS["prod384"]
    w = gi.make_workload(base, n=n)
    g = w.grid
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, precision=G.MIXED, safety=0.9)
    r.set_x(cuda(w.x0))
    r.set_B0(cuda(w.B0))
    E = [r.energy()]
    xi0 = r.forcefree_err()[0]
    for _ in range(49):
        st = r.step(200)
        assert st["status"] == 0
        E.append(r.energy())
    E = np.array(E)
    # E_M never rises (FP64 sums of FP32 fields: allow rounding-level noise)
    assert np.all(np.diff(E) <= 1e-7 * E[0]) and E[-1] < E[0]
    assert r.forcefree_err()[0] < 0.1 * xi0
    # the last 200 steps: their schedule, then the adjoint along them
    xs = r.get_x()
    dts = G.relax_with_schedule(r, xs, 200)
    assert len(dts) == 200 and r.stats()["accepted"] == 200
    X = gi.nodes(g)
    which = [0, 5, 11]
    dk, dl = [], []
    for q in which:
        a, b = gi.twist_region_grad(X, *w.regions[q])
        dk.append(a)
        dl.append(b)
    dB = cuda(np.stack(dk + dl))
    del X, dk, dl
    vm, mum, _ = G.loss_and_field_gradient(r, xs, dts, 0, checkpoint_every=10)
    gm = G.param_contract(dB, mum).cpu().numpy()
    del r, mum
    torch.cuda.empty_cache()
    rf = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi)
    rf.set_B0(cuda(w.B0))
    vf, muf, _ = G.loss_and_field_gradient(rf, xs, dts, 0, checkpoint_every=10)
    gf = G.param_contract(dB, muf).cpu().numpy()
    del rf, muf, dB
    torch.cuda.empty_cache()
    assert np.all(np.isfinite(gm)) and np.abs(gf).max() > 0
    assert abs(vm - vf) <= 1e-6 * abs(vf), (vm, vf)
    assert np.abs(gm - gf).max() <= 1e-6 * np.abs(gf).max(), (gm, gf)
