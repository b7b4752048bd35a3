"""Write the golden fixtures of tests/golden/ from the FP64 oracle only.

tube16_relax.json: the 16^3 twisted-tube workload relaxed by 20
error-controlled Cash-Karp steps (section "Time Stepping", eq. "time
stepping"; tolerance 1e-7, first step 1e-3) with the mimetic current: the
accepted step sizes, counters, time, E_M (eq. "magnetic energy"), xi and
the positions of a few sample nodes.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import glemur_inputs as gi  # noqa: E402
import oracle as ora  # noqa: E402

SAMPLES = [(1, 1, 1), (5, 7, 8), (8, 8, 8), (14, 3, 11), (10, 12, 2)]


def tube16_relax():
    w = gi.make_workload("tube", n=16)
    g = w.grid
    x, dt_next, log, st, rc = ora.relax(g, w.x0, w.B0, 20, 1e-3)
    assert rc == ora.OK
    E, _ = ora.energy(g, x, w.B0)
    xi, xi_sin, _ = ora.forcefree(g, x, w.B0)
    return {
        "workload": "tube, 16^3 nodes on [-1,1]^3, x = X",
        "steps": 20, "lambda0": 1e-7, "dt0": 1e-3,
        "accepted_dt": list(log), "rejected": st["rejected"], "t": st["t"],
        "dt_next": dt_next, "energy": E, "xi": xi, "xi_sin": xi_sin,
        "samples": [{"ijk": list(s), "x": [x[c, s[2], s[1], s[0]] for c in range(3)]}
                    for s in SAMPLES],
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "tube16_relax.json")
    with open(out, "w") as f:
        json.dump(tube16_relax(), f, indent=1)
    print(out)
