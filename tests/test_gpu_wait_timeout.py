"""Failure detection on the GPU without a fault: the mixed-precision
mimetic stages wait for their TMA tiles on shared-memory barriers with a
time limit.  GLEMUR_TEST_TMA_TIMEOUT=1 makes the prologue's tile wait also
wait on a barrier that no copy completes (=2: the first wait inside the
plane loop, which needs CTAs of at least two z-planes), so the wait gives
up after half a second; the kernel raises a flag, lets its own copies land
and returns, and the step control turns the flag into GLEMUR_ERR_TIMEOUT.
The device stays usable: a context created afterwards without the hook
matches the oracle."""
import time

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


def case():
    g = gi.Grid(64, 20, 8)
    X = gi.nodes(g)
    return g, gi.predistort(X, 2), gi.braid_field(X, gi.braid_regions(6, None, True))


def make(G, g, x0, B0):
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, precision=G.MIXED)
    r.set_x(torch.from_numpy(x0).cuda())
    r.set_B0(torch.from_numpy(B0).cuda())
    return r


@pytest.mark.parametrize("where", ["1", "2"], ids=["prologue", "plane-loop"])
def test_tile_wait_timeout_is_reported(G, monkeypatch, where):
    g, x0, B0 = case()
    monkeypatch.setenv("GLEMUR_TEST_TMA_TIMEOUT", where)
    # four z-planes per CTA, so every CTA reaches the loop's first wait
    monkeypatch.setenv("GLEMUR_KZ", "4")
    r = make(G, g, x0, B0)
    t0 = time.time()
    with pytest.raises(G.GlemurError) as err:
        r.step(1)
    assert err.value.code == -8
    assert time.time() - t0 < 60
    st = r.stats()
    assert st["status"] == -8 and st["accepted"] == 0
    # the state did not advance and the context reports the same status again
    with pytest.raises(G.GlemurError):
        r.step(1)
    del r
    monkeypatch.delenv("GLEMUR_TEST_TMA_TIMEOUT")
    monkeypatch.delenv("GLEMUR_KZ")
    r2 = make(G, g, x0, B0)
    u = r2.velocity().cpu().numpy()
    u_ref, _ = ora.velocity(g, x0, B0, 0)
    assert np.abs(u - u_ref).max() < 2e-4 * np.abs(u_ref).max()
    st = r2.step(2)
    assert st["accepted"] == 2 and st["status"] == 0
