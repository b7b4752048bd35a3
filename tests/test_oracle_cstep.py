"""Pins of the complex-step derivative oracle (glemur_oracle_cstep.c).

Its real part must reproduce the real oracle bit for bit, and Im(f)/h must
be the derivative: checked against closed forms (E_M exactly quadratic in a
field amplitude on a fixed grid; a uniform field's energy scaling) and
against central differences of the real oracle.
"""
import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora

H = ora.CSTEP_H


def test_real_part_reproduces_the_real_oracle():
    w = gi.make_workload("braid", n=10)
    u, _ = ora.velocity(w.grid, w.x0, w.B0)
    uc, _ = ora.cs_velocity(w.grid, w.x0, w.B0)
    assert np.array_equal(uc.real, u) and np.all(uc.imag == 0)
    dts = [2e-3, 3e-3]
    x = w.x0
    for dt in dts:
        x, _, _ = ora.step_fixed(w.grid, x, w.B0, dt)
    E_ref, _ = ora.energy(w.grid, x, w.B0)
    E, xc, rc = ora.cs_relax_loss(w.grid, w.x0, w.B0, dts, ora.LOSS_ENERGY)
    assert rc == ora.OK and np.array_equal(xc.real, x)
    assert E.real == E_ref
    xi_ref, _, _ = ora.forcefree(w.grid, x, w.B0)
    xi, _, _ = ora.cs_relax_loss(w.grid, w.x0, w.B0, dts, ora.LOSS_XI)
    assert abs(xi.real - xi_ref) < 1e-15 * xi_ref


def test_energy_is_quadratic_in_a_twist_amplitude():
    """On a fixed grid B is linear in B0, so E_M(k) = a + b k + c k^2
    exactly; three real evaluations give b + 2 c k0, which the complex step
    must reproduce."""
    g = gi.Grid(9, 10, 11)
    X = gi.nodes(g)
    x = gi.predistort(X, 4)

    def B0(k):
        return gi.braid_field(X, [(0.1, -0.2, 0.0, k, 0.5, 0.6)])

    Es = [ora.energy(g, x, B0(k))[0] for k in (-1.0, 0.0, 1.0)]
    c2 = (Es[0] + Es[2] - 2 * Es[1]) / 2
    b1 = (Es[2] - Es[0]) / 2
    k0 = 0.7
    exact = b1 + 2 * c2 * k0
    E, _, _ = ora.cs_relax_loss(g, x, B0(k0 + 1j * H), [], ora.LOSS_ENERGY)
    assert abs(E.imag / H - exact) < 1e-12 * abs(exact)


def test_uniform_field_energy_scales_quadratically_through_steps():
    """A uniform field on an affine grid is stationary, so after any steps
    E(s B0) = s^2 E(B0) and dE/ds = 2 s E(B0)."""
    g = gi.Grid(7, 7, 7)
    X = gi.nodes(g)
    A = np.array([[1.05, 0.1, 0.0], [0.0, 0.95, 0.05], [0.02, 0.0, 1.1]])
    x = np.einsum("ab,b...->a...", A, X)
    Bu = gi.uniform_field(g, (0.2, 0.1, 1.0))
    s = 1.3
    E1, _, _ = ora.cs_relax_loss(g, x, Bu, [1e-3, 1e-3], ora.LOSS_ENERGY)
    Es, _, _ = ora.cs_relax_loss(g, x, (s + 1j * H) * Bu, [1e-3, 1e-3], ora.LOSS_ENERGY)
    assert abs(Es.imag / H - 2 * s * E1.real) < 1e-12 * E1.real


@pytest.mark.parametrize("loss", [ora.LOSS_ENERGY, ora.LOSS_XI])
def test_complex_step_matches_central_differences(loss):
    """d loss / d theta after a few steps at a frozen schedule: complex step
    against central differences of the real oracle (h = 1e-5, truncation
    O(h^2))."""
    theta0 = np.array([1.0, -1.0, 0.3, 0.3])        # (k_0, k_1, l_0, l_1)
    g = gi.Grid(10, 10, 10)
    X = gi.nodes(g)
    x0 = gi.predistort(X, 2)

    def B0(th):
        regs = [(0.3, 0.0, -0.3, th[0], th[2], 0.4), (-0.3, 0.0, 0.3, th[1], th[3], 0.4)]
        return gi.braid_field(X.astype(complex) if np.iscomplexobj(th) else X, regs)

    dts = [1e-3, 2e-3, 2e-3]

    def real_loss(th):
        x = x0
        for dt in dts:
            x, _, _ = ora.step_fixed(g, x, B0(th), dt)
        if loss == ora.LOSS_ENERGY:
            return ora.energy(g, x, B0(th))[0]
        return ora.forcefree(g, x, B0(th))[0]

    for p in range(4):
        e = np.zeros(4)
        e[p] = 1.0
        L, _, rc = ora.cs_relax_loss(g, x0, B0(theta0 + 1j * H * e), dts, loss)
        assert rc == ora.OK
        d_cs = L.imag / H
        hh = 1e-5
        d_fd = (real_loss(theta0 + hh * e) - real_loss(theta0 - hh * e)) / (2 * hh)
        assert abs(d_cs - d_fd) < 1e-6 * max(abs(d_cs), 1e-3), (p, d_cs, d_fd)
