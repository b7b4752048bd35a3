"""Oracle runs that tests hand to spawned worker processes (plain C on the
host, no GPU): kept apart from the test modules so that a worker imports
only the oracle and the input generators."""
import numpy as np

import glemur_inputs as gi
import oracle as ora


def cs_braid_direction(job):
    """Complex-step derivative of the braid workload's loss along a
    direction in its 12 parameters: job = (nodes per axis, step sizes,
    direction, loss, h).  Returns (loss, directional derivative, status)."""
    n, dts, direction, loss, h = job
    w = gi.make_workload("adjoint", n=n)
    X = gi.nodes(w.grid)
    m = len(w.regions)
    th = np.array(w.theta, dtype=np.complex128) + 1j * h * np.asarray(direction)
    regs = [(rr[0], rr[1], rr[2], th[i], th[m + i], rr[5]) for i, rr in enumerate(w.regions)]
    Lc, _, rc = ora.cs_relax_loss(w.grid, w.x0, gi.braid_field(X, regs), dts, loss)
    return Lc.real, Lc.imag / h, rc
