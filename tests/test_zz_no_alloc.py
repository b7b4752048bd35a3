"""glemur_energy_static: the energy reduction for callers that cannot
allocate device memory (a host framework owning the whole device pool, or
code that must avoid cudaMalloc's implicit synchronisation).  Its scratch is
a static device array, so it takes no workspace and no context.

This file is collected last so that a failure here cannot hide the rest of
the GPU suite in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import glemur_inputs as gi
import oracle as ora

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_0942_gb300.glemur as g
    return g.lib()


def _energy_static(L, g, x_dev, B0_dev, E_dev):
    lo = (ctypes.c_double * 3)(*g.lo)
    hi = (ctypes.c_double * 3)(*g.hi)
    stream = torch.cuda.current_stream().cuda_stream
    return L.glemur_energy_static(g.nx, g.ny, g.nz, lo, hi, ctypes.c_void_p(x_dev.data_ptr()),
                                  ctypes.c_void_p(B0_dev.data_ptr()),
                                  ctypes.c_void_p(E_dev.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("dims", [(40, 33, 29), (16, 16, 16)])
def test_energy_static_matches_energy_twice(L, dims):
    """Two calls in a row through the C ABI agree with glemur_energy (the
    context-and-workspace entry point) to the FP64 energy tolerance used by
    the parity suite (1e-13 relative)."""
    import paper_1405_0942_gb300 as G
    g = gi.Grid(*dims)
    X = gi.nodes(g)
    x0 = gi.predistort(X, 2)
    B0 = gi.braid_field(X, gi.braid_regions(6, None, True))
    x_dev = torch.from_numpy(x0).cuda()
    B0_dev = torch.from_numpy(B0).cuda()
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi)
    r.set_x(x_dev)
    r.set_B0(B0_dev)
    E_ref = r.energy()
    for _ in range(2):
        E_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _energy_static(L, g, x_dev, B0_dev, E_dev) == 0
        E = float(E_dev.item())
        assert abs(E - E_ref) < 1e-13 * E_ref, (E, E_ref)


def test_energy_static_matches_oracle_and_allocates_nothing(L):
    """The entry point's own Jacobian and energy kernels against the FP64
    oracle's eq. "magnetic energy" (1e-13 relative), on a ragged grid with
    a pre-distorted interior; after a first call (which may load the
    library's device code), further calls leave the device's free memory
    unchanged."""
    g = gi.Grid(37, 21, 26)
    X = gi.nodes(g)
    x0 = gi.predistort(X, 4) + 0.01 * np.sin(2.0 * X[[1, 2, 0]])
    B0 = gi.braid_field(X, gi.braid_regions(6, 7, False)) + 0.1 * gi.abc_field(X)
    E_ref, rc = ora.energy(g, x0, B0)
    assert rc == ora.OK
    x_dev = torch.from_numpy(x0).cuda()
    B0_dev = torch.from_numpy(B0).cuda()
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _energy_static(L, g, x_dev, B0_dev, E_dev) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        E_dev.fill_(float("nan"))
        assert _energy_static(L, g, x_dev, B0_dev, E_dev) == 0
        torch.cuda.synchronize()
        assert abs(float(E_dev.item()) - E_ref) < 1e-13 * E_ref
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_energy_static_rejects_oversize_and_bad_args(L):
    big = gi.Grid(257, 256, 256)          # 16,842,752 nodes > 2^24
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _energy_static(L, big, dummy, dummy, dummy) == -7
    assert L.glemur_strerror(-7) == b"grid larger than the fixed scratch supports"
    small = gi.Grid(2, 5, 5)
    assert _energy_static(L, small, dummy, dummy, dummy) == -1
