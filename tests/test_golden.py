"""Golden fixture tests/golden/tube16_relax.json (written by
tests/golden/make_golden.py from the oracle only): the oracle must keep
reproducing it, and the GPU library must match it within the FP64 parity
tolerances without running the oracle.

The oracle's own check allows last-bit differences: the seeded inputs go
through numpy's exp and sin, whose results may differ by an ulp between CPU
architectures, and the step-size law dt' = dt (Lambda0/Lambda)^0.2 passes on
the relative rounding of the small error norm Lambda."""
import json
import os

import numpy as np
import pytest

import glemur_inputs as gi

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tube16_relax.json")


def load():
    with open(GOLD) as f:
        return json.load(f)


def test_oracle_reproduces_golden():
    import oracle as ora
    gold = load()
    w = gi.make_workload("tube", n=16)
    x, dt_next, log, st, rc = ora.relax(w.grid, w.x0, w.B0, gold["steps"], gold["dt0"])
    assert rc == ora.OK
    assert st["rejected"] == gold["rejected"] and len(log) == len(gold["accepted_dt"])
    assert np.allclose(log, gold["accepted_dt"], rtol=1e-9, atol=0)
    assert abs(ora.energy(w.grid, x, w.B0)[0] - gold["energy"]) <= 1e-13 * gold["energy"]
    for s in gold["samples"]:
        i, j, k = s["ijk"]
        assert np.abs(x[:, k, j, i] - np.array(s["x"])).max() <= 1e-12


@pytest.mark.gpu
def test_gpu_matches_golden():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_0942_gb300 as G
    gold = load()
    w = gi.make_workload("tube", n=16)
    g = w.grid
    r = G.Relaxation(g.nx, g.ny, g.nz, lambda0=gold["lambda0"], dt0=gold["dt0"])
    r.set_x(torch.from_numpy(w.x0).cuda())
    r.set_B0(torch.from_numpy(w.B0).cuda())
    st = r.step(gold["steps"])
    assert st["rejected"] == gold["rejected"]
    assert abs(st["t"] - gold["t"]) < 1e-9 * gold["t"]
    x = r.get_x().cpu().numpy()
    for s in gold["samples"]:
        i, j, k = s["ijk"]
        assert np.abs(x[:, k, j, i] - np.array(s["x"])).max() < 1e-10
    assert abs(r.energy() - gold["energy"]) < 1e-12 * gold["energy"]
    xi, xis = r.forcefree_err()
    assert abs(xi - gold["xi"]) < 1e-8 * gold["xi"]
