"""Programmatic dependent launch changes when a kernel may start, never
what it computes: attempts run with ordinary launches (GLEMUR_PDL=0, read
once per process, so in a child process) give bit-identical positions,
step sizes and diagnostics."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # (nx, ny, nz, precision, curl): FP64 two-pass, mixed TMA tiles,
    (20, 18, 16, 0, 0),  # mixed register-staged tiles, FP64 direct current
    (48, 24, 20, 1, 0),
    (21, 13, 17, 1, 0),
    (21, 13, 17, 0, 1),
]

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1405_0942_gb300 as G
import glemur_inputs as gi
out = {}
for nx, ny, nz, prec, curl in json.loads(sys.argv[2]):
    g = gi.Grid(nx, ny, nz)
    X = gi.nodes(g)
    x0 = gi.predistort(X, 2)
    B0 = gi.braid_field(X, gi.braid_regions(6, None, True))
    r = G.Relaxation(nx, ny, nz, precision=prec, curl=curl, diag_each_attempt=1)
    r.set_x(torch.from_numpy(x0).cuda())
    r.set_B0(torch.from_numpy(B0).cuda())
    r.attempts(6)
    x = r.get_x().cpu().numpy()
    st = r.stats()
    np.save(sys.argv[3] + f"_{nx}_{ny}_{nz}_{prec}_{curl}.npy", x)
    out[f"{nx}_{ny}_{nz}_{prec}_{curl}"] = {k: st[k] for k in ("accepted", "rejected", "dt", "t", "lam", "energy", "xi")}
print(json.dumps(out))
"""


def _run(env_pdl, tmp_path, tag):
    env = dict(os.environ, GLEMUR_PDL=env_pdl)
    res = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(CASES),
                          str(tmp_path / tag)], env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def test_pdl_and_ordinary_launches_agree_bit_for_bit(tmp_path):
    on = _run("1", tmp_path, "on")
    off = _run("0", tmp_path, "off")
    assert on == off
    for nx, ny, nz, prec, curl in CASES:
        key = f"{nx}_{ny}_{nz}_{prec}_{curl}"
        a = np.load(tmp_path / f"on_{key}.npy")
        b = np.load(tmp_path / f"off_{key}.npy")
        assert np.array_equal(a, b), key
