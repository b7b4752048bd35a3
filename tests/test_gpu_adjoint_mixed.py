"""The adjoint on mixed-precision contexts: the reverse kernels run in FP64
arithmetic along the FP32-stored trajectory (the stage recompute uses the
mixed stage kernels).  Over the last steps of a run -- the state after some
controlled steps is the start, the next steps' sizes are frozen -- the
parameter gradient of a mixed context agrees with that of an FP64 context
replaying the same schedule from the same state, to the mixed path's
accuracy; on the 128^3 braid (10 twist regions) and on the 384^3
production workload (12 regions + ABC), the configuration whose adjoint
covers its last steps in mixed precision."""
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


def param_grad_subset(X, regions, which):
    """dB0/dtheta for the amplitudes and widths of the regions `which`."""
    dk, dl = [], []
    for q in which:
        a, b = gi.twist_region_grad(X, *regions[q])
        dk.append(a)
        dl.append(b)
    return np.stack(dk + dl)


@pytest.mark.parametrize("name,warm,steps,which,tol",
                         [("braid128", 10, 20, list(range(10)), 1e-4),
                          ("prod384", 5, 8, [0, 5, 11], 1e-3)],
                         ids=["braid128", "prod384"])
@pytest.mark.parametrize("loss", [0, 1], ids=["energy", "xi"])
def test_mixed_adjoint_matches_fp64(G, name, warm, steps, which, tol, loss):
    base, n, _ = gi.WORKLOADS[name]
    w = gi.make_workload(base, n=n)
    g = w.grid
    X = gi.nodes(g)
    dB = cuda(param_grad_subset(X, w.regions, which))
    rm = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, precision=G.MIXED, safety=0.9)
    rm.set_x(cuda(w.x0))
    rm.set_B0(cuda(w.B0))
    rm.step(warm)
    xs = rm.get_x()
    dts = G.relax_with_schedule(rm, xs, steps)
    vm, mum, _ = G.loss_and_field_gradient(rm, xs, dts, loss, checkpoint_every=4)
    gm = G.param_contract(dB, mum).cpu().numpy()
    del rm, mum
    torch.cuda.empty_cache()
    rf = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi)
    rf.set_B0(cuda(w.B0))
    vf, muf, _ = G.loss_and_field_gradient(rf, xs, dts, loss, checkpoint_every=4)
    gf = G.param_contract(dB, muf).cpu().numpy()
    del rf, muf, dB
    torch.cuda.empty_cache()
    assert abs(vm - vf) <= (1e-6 if loss == 0 else 1e-3) * abs(vf), (vm, vf)
    err = np.abs(gm - gf).max() / np.abs(gf).max()
    assert err < tol, (err, gm, gf)
