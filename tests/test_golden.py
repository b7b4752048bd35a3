"""Golden fixture tests/golden/tube16_relax.json (written by
tests/golden/make_golden.py from the oracle only): the oracle must keep
reproducing it exactly, and the GPU library must match it within the FP64
parity tolerances without running the oracle."""
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
    assert list(log) == gold["accepted_dt"] and st["rejected"] == gold["rejected"]
    assert ora.energy(w.grid, x, w.B0)[0] == gold["energy"]
    for s in gold["samples"]:
        i, j, k = s["ijk"]
        assert [x[c, k, j, i] for c in range(3)] == s["x"]


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
