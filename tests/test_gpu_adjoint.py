"""GPU adjoint (reverse mode of the relaxation) against the complex-step
oracle and central finite differences.

The oracle side is glemur_oracle_cstep.c: the forward method in complex
arithmetic, whose Im(output)/h is the exact directional derivative.  The
adjoint is checked through dot products: <lam, v> = <lam_next, (dx'/dx) v>
and <mu, w> = <lam_next, (dx'/dB0) w> for random directions v, w.
Tolerance: both sides are FP64 with O(10^3) operations per node and step;
agreement is required to 1e-9 relative for single steps and losses, and the
parameter gradient to 1e-6 relative of central differences (h = 1e-6
relative), the target the method states.
"""
import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
H = ora.CSTEP_H


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_0942_gb300 as pkg
    pkg.lib()
    return pkg


def case(nx, ny, nz, seed=2, n_regions=6):
    g = gi.Grid(nx, ny, nz)
    X = gi.nodes(g)
    regs = gi.braid_regions(n_regions, None, True, l=0.35, L=0.3)
    return g, X, gi.predistort(X, seed), regs


def interior_mask(g):
    m = np.zeros((3, g.nz, g.ny, g.nx))
    m[:, 1:-1, 1:-1, 1:-1] = 1.0
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relax_for(G, g, x0, B0, **kw):
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi, **kw)
    r.set_x(cuda(x0))
    r.set_B0(cuda(B0))
    return r


def test_vjp_step_dot_products(G):
    g, X, x0, regs = case(12, 11, 13)
    B0 = gi.braid_field(X, regs)
    dt = 3e-3
    rng = np.random.default_rng(0)
    lam_next = rng.standard_normal(x0.shape) * interior_mask(g)
    v = rng.standard_normal(x0.shape) * interior_mask(g)
    w = rng.standard_normal(B0.shape)
    _, x1v, rc = ora.cs_relax_loss(g, x0 + 1j * H * v, B0, [dt])
    assert rc == ora.OK
    _, x1w, _ = ora.cs_relax_loss(g, x0, B0 + 1j * H * w, [dt])
    Jv, Jw = x1v.imag / H, x1w.imag / H
    r = relax_for(G, g, x0, B0)
    lam = torch.zeros_like(cuda(x0))
    mu = torch.zeros_like(lam)
    r.vjp_step(dt, cuda(lam_next), lam, mu)
    lam, mu = lam.cpu().numpy(), mu.cpu().numpy()
    lhs_x, rhs_x = (lam * v).sum(), (lam_next * Jv).sum()
    lhs_b, rhs_b = (mu * w).sum(), (lam_next * Jw).sum()
    assert abs(lhs_x - rhs_x) < 1e-9 * abs(rhs_x), (lhs_x, rhs_x)
    assert abs(lhs_b - rhs_b) < 1e-9 * abs(rhs_b), (lhs_b, rhs_b)
    # boundary positions are not variables
    lb = lam.copy()
    lb[:, 1:-1, 1:-1, 1:-1] = 0
    assert np.all(lb == 0)


@pytest.mark.parametrize("loss", [0, 1], ids=["energy", "xi"])
def test_loss_gradient_dot_products(G, loss):
    g, X, x0, regs = case(13, 12, 11)
    B0 = gi.braid_field(X, regs)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(x0.shape) * interior_mask(g)
    w = rng.standard_normal(B0.shape)
    Lv, _, _ = ora.cs_relax_loss(g, x0 + 1j * H * v, B0, [], loss)
    Lw, _, _ = ora.cs_relax_loss(g, x0, B0 + 1j * H * w, [], loss)
    r = relax_for(G, g, x0, B0)
    lam = torch.zeros_like(cuda(x0))
    mu = torch.zeros_like(lam)
    value = r.loss_grad(loss, lam, mu)
    assert abs(value - Lv.real) < 1e-12 * abs(Lv.real)
    dv = (lam.cpu().numpy() * v).sum()
    dw = (mu.cpu().numpy() * w).sum()
    assert abs(dv - Lv.imag / H) < 1e-9 * abs(Lv.imag / H)
    assert abs(dw - Lw.imag / H) < 1e-9 * abs(Lw.imag / H)


@pytest.mark.parametrize("loss", [0, 1], ids=["energy", "xi"])
def test_parameter_gradient_through_steps(G, loss):
    """dL/dtheta for the 12 braid parameters (6 amplitudes, 6 widths) after
    12 steps with checkpoints every 5: adjoint vs complex-step oracle and vs
    GPU central differences, all at the same frozen step-size schedule."""
    g, X, x0, regs = case(14, 14, 16)
    B0 = gi.braid_field(X, regs)
    x_ref, _, dts, st, rc = ora.relax(g, x0, B0, 12, 2e-3)
    assert rc == ora.OK
    r = relax_for(G, g, x0, B0)
    value, mu, _ = G.loss_and_field_gradient(r, cuda(x0), dts, loss, checkpoint_every=5)
    dB = cuda(gi.braid_field_param_grad(X, regs))
    grad = G.param_contract(dB, mu).cpu().numpy()
    theta = np.array([rr[3] for rr in regs] + [rr[4] for rr in regs])

    def regions(th):
        m = len(regs)
        return [(rr[0], rr[1], rr[2], th[i], th[m + i], rr[5]) for i, rr in enumerate(regs)]

    for p in range(len(theta)):
        e = np.zeros(len(theta))
        e[p] = 1.0
        Bc = gi.braid_field(X, regions(theta + 1j * H * e))
        Lc, _, _ = ora.cs_relax_loss(g, x0, Bc, dts, loss)
        d_or = Lc.imag / H
        assert abs(grad[p] - d_or) < 1e-8 * max(abs(d_or), 1e-6 * abs(Lc.real)), (p, grad[p], d_or)
        hh = 1e-6 * abs(theta[p])
        Lp, Lm = [], []
        for sgn, out in ((1, Lp), (-1, Lm)):
            r.set_B0(cuda(gi.braid_field(X, regions(theta + sgn * hh * e))))
            r.set_x(cuda(x0))
            for dt in dts:
                r.step_fixed(dt)
            if loss == 0:
                out.append(r.energy())
            else:
                out.append(r.forcefree_err()[0])
        d_fd = (Lp[0] - Lm[0]) / (2 * hh)
        assert abs(grad[p] - d_fd) < 1e-6 * max(abs(grad[p]), 1e-6 * abs(Lc.real)), \
            (p, grad[p], d_fd)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n,every", [(12, 5), (7, 7), (3, 10), (0, 4)],
                         ids=["12by5", "7by7", "3by10", "none"])
def test_native_segment_matches_the_orchestrated_sweep(G, precision, n, every):
    """glemur_adjoint_segment (checkpoints, recompute and reverse steps in
    the library) against the same algorithm orchestrated call by call
    (forward_checkpoints + reverse_sweep over glemur_get_state / set_state /
    step_fixed / vjp_step / loss_grad): the same kernels in the same order,
    so loss, dL/dB0 and dL/dx0 agree bit for bit, for segment lengths that
    do and do not divide the step count, a single partial segment and no
    steps at all."""
    g, X, x0, regs = case(14, 13, 15)
    B0 = gi.braid_field(X, regs)
    dts = [2e-3 * (1.0 + 0.1 * (i % 3)) for i in range(n)]
    r = relax_for(G, g, x0, B0, precision=precision)
    for loss in (0, 1):
        v1, mu1, lam1 = r.adjoint_segment(cuda(x0), dts, loss, every)
        ck = G.forward_checkpoints(r, cuda(x0), dts, every)
        v2, mu2, lam2 = G.reverse_sweep(r, ck, dts, loss, every)
        assert v1 == v2
        assert torch.equal(mu1, mu2) and torch.equal(lam1, lam2)
        assert float(mu1.abs().max()) > 0


def test_native_segment_argument_errors(G):
    g, X, x0, regs = case(8, 8, 8)
    r = relax_for(G, g, x0, gi.braid_field(X, regs))
    with pytest.raises(G.GlemurError):
        r.adjoint_segment(cuda(x0), [1e-3, -1.0], 0, 2)      # a step size <= 0
    with pytest.raises(G.GlemurError):
        r.adjoint_segment(cuda(x0), [1e-3], 5, 2)            # no such loss


def test_autograd_function(G):
    """torch.autograd through RelaxationFieldLoss gives the field gradient."""
    g, X, x0, regs = case(10, 10, 10)
    B0 = cuda(gi.braid_field(X, regs)).requires_grad_(True)
    r = G.Relaxation(g.nx, g.ny, g.nz)
    dts = [2e-3] * 4
    L = G.RelaxationFieldLoss.apply(r, B0, cuda(x0), dts, 0, 2)
    L.backward()
    _, mu, _ = G.loss_and_field_gradient(r, cuda(x0), dts, 0, checkpoint_every=3)
    assert torch.allclose(B0.grad, mu, rtol=1e-12, atol=0)


@pytest.mark.parametrize("loss", [0, 1], ids=["energy", "xi"])
def test_autograd_over_parameters(G, loss):
    """RelaxationLoss is an autograd.Function of theta (the 6 amplitudes and
    6 widths): forward only relaxes and checkpoints (no reverse step runs),
    returns the loss of the final state; backward runs the reverse sweep and
    contracts with dB0/dtheta on the device -- the same gradient as the
    explicit adjoint and contraction."""
    g, X, x0, regs = case(12, 11, 13)
    m = len(regs)
    r = G.Relaxation(g.nx, g.ny, g.nz)
    dts = [2e-3] * 7

    def field(th):
        t = th.cpu().numpy()
        rg = [(rr[0], rr[1], rr[2], t[i], t[m + i], rr[5]) for i, rr in enumerate(regs)]
        return cuda(gi.braid_field(X, rg)), cuda(gi.braid_field_param_grad(X, rg))

    theta = torch.tensor([rr[3] for rr in regs] + [rr[4] for rr in regs], dtype=torch.float64,
                         device="cuda", requires_grad=True)
    calls = []
    orig = r.vjp_step
    r.vjp_step = lambda *a: (calls.append(1), orig(*a))[1]
    L = G.RelaxationLoss.apply(r, theta, field, cuda(x0), dts, loss, 3)
    assert not calls                                  # forward: no reverse work
    r.set_x(cuda(x0))
    for dt in dts:
        r.step_fixed(dt)
    ref_val = r.energy() if loss == 0 else r.forcefree_err()[0]
    assert float(L.detach()) == pytest.approx(ref_val, rel=1e-14)
    (2.0 * L).backward()
    assert len(calls) == len(dts)
    B0, dB = field(theta.detach())
    r.set_B0(B0)
    value, mu, _ = G.loss_and_field_gradient(r, cuda(x0), dts, loss, checkpoint_every=3)
    want = 2.0 * G.param_contract(dB, mu)
    assert torch.allclose(theta.grad, want, rtol=1e-12, atol=0)


def test_adjoint_96_cubed_500_steps_vs_fd(G):
    """The 96^3 braid workload, 500 error-controlled FP64 steps (schedule
    recorded, then frozen), checkpoints every 50: gradient of the final
    energy with respect to the 6 twist amplitudes and 6 widths against
    central differences.  At this size E_M carries ~1e-12 of rounding noise,
    so differences with h = 1e-6 are noise-limited (~1e-4 relative); a step
    study (h = 1e-7 .. 1e-3) converges to the adjoint, and h = 1e-3 relative
    (truncation ~1e-7) is used."""
    w = gi.make_workload("adjoint")
    g = w.grid
    X = gi.nodes(g)
    r = relax_for(G, g, w.x0, w.B0)
    x0 = cuda(w.x0)
    dts = G.relax_with_schedule(r, x0, 500)
    value, mu, _ = G.loss_and_field_gradient(r, x0, dts, 0, checkpoint_every=50)
    grad = G.param_contract(cuda(gi.braid_field_param_grad(X, w.regions)), mu).cpu().numpy()
    theta = np.array(w.theta)
    m = len(w.regions)
    for p in range(len(theta)):
        hh = 1e-3 * abs(theta[p])
        vals = []
        for sgn in (1, -1):
            th = theta.copy()
            th[p] += sgn * hh
            regs = [(rr[0], rr[1], rr[2], th[i], th[m + i], rr[5]) for i, rr in enumerate(w.regions)]
            r.set_B0(cuda(gi.braid_field(X, regs)))
            r.set_x(x0)
            for dt in dts:
                r.step_fixed(dt)
            vals.append(r.energy())
        d_fd = (vals[0] - vals[1]) / (2 * hh)
        assert abs(grad[p] - d_fd) < 1e-6 * max(abs(grad[p]), 1e-7 * value), (p, grad[p], d_fd)


def _argmax_xi(G, r, g, B0):
    """Interior node of max |J x B| / B^2 of the relaxation's state: u = J x B
    from the library, B the oracle's pull-back of B0 on the same positions."""
    u = r.velocity().cpu().numpy()
    x = r.get_x().cpu().numpy()
    B, _, _ = ora.pullback(g, x, B0)
    q = np.sqrt((u * u).sum(0)) / (B * B).sum(0)
    q[[0, -1], :, :] = 0
    q[:, [0, -1], :] = 0
    q[:, :, [0, -1]] = 0
    return np.unravel_index(np.argmax(q), q.shape)


def test_adjoint_96_cubed_500_steps_xi_vs_fd(G):
    """The 96^3 braid, 500 error-controlled steps (schedule frozen),
    checkpoints every 50: gradient of the final force-free error xi (taken at
    its argmax node) with respect to the 12 parameters against central
    differences of fourth order, (8 (L(h) - L(-h)) - (L(2h) - L(-2h))) / 12h
    at h = 1e-3 relative.  xi (a maximum of second differences of x)
    carries ~1e-12 relative rounding noise at this size, so small steps are
    noise-limited (at h = 1e-4 the error of an amplitude component was
    1.8e-6), while second-order differences at h = 1e-3 keep 2.5e-6 of
    truncation error for the widths; the fourth-order formula removes that
    at the larger step.  xi is a maximum: its difference quotient is the
    derivative only while the argmax node stays put, so the node is checked
    at theta and at every perturbed theta."""
    w = gi.make_workload("adjoint")
    g = w.grid
    X = gi.nodes(g)
    r = relax_for(G, g, w.x0, w.B0)
    x0 = cuda(w.x0)
    dts = G.relax_with_schedule(r, x0, 500)
    value, mu, _ = G.loss_and_field_gradient(r, x0, dts, 1, checkpoint_every=50)
    grad = G.param_contract(cuda(gi.braid_field_param_grad(X, w.regions)), mu).cpu().numpy()
    r.set_x(x0)
    for dt in dts:
        r.step_fixed(dt)
    node0 = _argmax_xi(G, r, g, w.B0)
    theta = np.array(w.theta)
    m = len(w.regions)
    for p in range(len(theta)):
        hh = 1e-3 * abs(theta[p])
        vals = {}
        for mult in (1, -1, 2, -2):
            th = theta.copy()
            th[p] += mult * hh
            regs = [(rr[0], rr[1], rr[2], th[i], th[m + i], rr[5])
                    for i, rr in enumerate(w.regions)]
            B0p = gi.braid_field(X, regs)
            r.set_B0(cuda(B0p))
            r.set_x(x0)
            for dt in dts:
                r.step_fixed(dt)
            vals[mult] = r.forcefree_err()[0]
            assert _argmax_xi(G, r, g, B0p) == node0, (p, mult)
        d_fd = (8.0 * (vals[1] - vals[-1]) - (vals[2] - vals[-2])) / (12.0 * hh)
        assert abs(grad[p] - d_fd) < 1e-6 * max(abs(grad[p]), 1e-7 * value), \
            (p, grad[p], d_fd)
    r.set_B0(cuda(w.B0))


def test_adjoint_96_cubed_vs_complex_step_oracle(G):
    """At 96^3 over the first 20 steps of the error-controlled schedule: the
    GPU parameter gradient of both losses, dotted with a random direction in
    theta, against the complex-step derivative of the FP64 oracle along that
    direction (exact to rounding), within 1e-8."""
    import multiprocessing as mp
    w = gi.make_workload("adjoint")
    g = w.grid
    X = gi.nodes(g)
    r = relax_for(G, g, w.x0, w.B0)
    x0 = cuda(w.x0)
    dts = G.relax_with_schedule(r, x0, 20)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(12)
    jobs = [(96, list(dts), v, loss, H) for loss in (0, 1)]
    from oracle_jobs import cs_braid_direction
    with mp.get_context("spawn").Pool(2) as pool:
        res = pool.map(cs_braid_direction, jobs)
    dB = cuda(gi.braid_field_param_grad(X, w.regions))
    for loss, (Lr, dL, rc) in zip((0, 1), res):
        assert rc == ora.OK
        value, mu, _ = G.loss_and_field_gradient(r, x0, dts, loss, checkpoint_every=50)
        grad = G.param_contract(dB, mu).cpu().numpy()
        assert abs(grad @ v - dL) < 1e-8 * abs(dL), (loss, grad @ v, dL)
        # after 20 steps the two trajectories differ at ~1e-12 in x, which
        # the loss (through derivatives of x) amplifies by ~1/h
        assert abs(value - Lr) < 1e-9 * abs(Lr)
