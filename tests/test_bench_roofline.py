"""The benchmark's roofline arithmetic on synthetic timings (no GPU):
achieved = algorithmic bytes (FP64: flops) of the six stage launches over
the whole-attempt time, frac = achieved / peak, stage shares from the
event-separated split."""
import numpy as np

import bench


class _G:
    def __init__(self, n):
        self.nx = self.ny = self.nz = n
        self.n_interior = (n - 2) ** 3


class _W:
    def __init__(self, n):
        self.grid = _G(n)


def test_mixed_roofline_is_bytes_over_whole_attempt():
    w = _W(128)
    whole = np.array([0.35, 0.35])                     # ms per attempt
    split = np.array([[0.06] * 6 + [0.01]] * 2)        # six stages + control
    r = bench.roofline_entry(whole, split, w, "braid128", "mixed", "mimetic", 6783.8, "measured")
    I = 126 ** 3
    gbs = 66.0 * I * 6 / (0.35e-3) / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert np.isclose(r["achieved"], gbs) and np.isclose(r["frac"], gbs / 6783.8)
    assert r["algorithmic_bytes_per_launch"] == 66.0 * I
    ent = bench.NCU_TRAFFIC.get(("braid128", "mixed", "mimetic"))
    fresh = ent is not None and ent[1] == bench.kernel_source_hash()
    assert r["traffic"] == (ent[0] if fresh else None)
    assert np.isclose(sum(r["stage_shares"]), 0.36 / 0.37, atol=1e-3)


def test_fp64_roofline_is_flops_against_the_fp64_rate():
    w = _W(64)
    whole = np.array([0.4])
    split = np.array([[0.07] * 6 + [0.01]])
    r = bench.roofline_entry(whole, split, w, "braid64", "fp64", "mimetic", 6783.8, "measured")
    I = 62 ** 3
    tf = bench.ALGO_FLOPS_F64["mimetic"] * I * 6 / 0.4e-3 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert np.isclose(r["achieved"], tf)
    assert np.isclose(r["frac"], tf * 1e12 / bench.FP64_PEAK_FLOPS)
    assert np.isclose(r["hbm_achieved_gbs"], 132.0 * I * 6 / 0.4e-3 / 1e9)


def test_workload_without_a_capture_reports_null_traffic():
    r = bench.roofline_entry(np.array([1.0]), np.array([[0.1] * 7]), _W(96), "adjoint96",
                             "mixed", "direct", 6783.8, "measured")
    assert r["traffic"] is None


def test_traffic_goes_null_when_the_kernels_change(monkeypatch):
    """A traffic figure is reported only with the kernel sources it was
    captured on: an entry carrying another source hash reads as null."""
    h = bench.kernel_source_hash()
    assert len(h) == 12
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("w40", "mixed", "mimetic"), (1.5e6, h))
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("w41", "mixed", "mimetic"), (1.5e6, "0" * 12))
    assert bench.ncu_traffic("w40", "mixed", "mimetic") == 1.5e6
    assert bench.ncu_traffic("w41", "mixed", "mimetic") is None


def test_nnn_roofline_uses_its_own_flop_count():
    r = bench.roofline_entry(np.array([1.0]), np.array([[0.15] * 6 + [0.01]]), _W(64),
                             "braid64", "fp64", "nnn", 6783.8, "measured")
    I = 62 ** 3
    assert np.isclose(r["achieved"], 729.0 * I * 6 / 1e-3 / 1e12)
    assert r["algorithmic_flops_per_launch"] == 729.0 * I


def test_traffic_table_covers_the_default_run_on_the_current_kernels():
    """Every stage-kernel roofline the default benchmark line carries (the
    headline and its comparison modes) has a traffic figure captured on the
    current stage-kernel sources, so none of them reports null."""
    h = bench.kernel_source_hash()
    modes = [("braid64", "fp64", "mimetic"), ("braid64", "mixed", "mimetic"),
             ("braid64", "fp64", "direct"), ("braid64", "mixed", "direct"),
             ("braid64", "fp64", "nnn"), ("periodic64", "fp64", "mimetic"),
             ("braid128", "mixed", "mimetic"), ("prod384", "mixed", "mimetic")]
    for m in modes:
        assert m in bench.NCU_TRAFFIC, m
        assert bench.NCU_TRAFFIC[m][1] == h, (m, bench.NCU_TRAFFIC[m][1], h)
        assert bench.ncu_traffic(*m) > 0
