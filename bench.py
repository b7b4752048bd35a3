"""Throughput of the Lagrangian magneto-frictional relaxation step on GB300.

A step is one Cash-Karp attempt of the whole hot path (six stages -- stage
input, Jacobian, pull-back, current, J x B; one fused kernel per stage in
mixed precision, two passes per stage in FP64 -- the fifth-order update
with its embedded error, and the step control) over the 64^3 braid
workload (6 twist regions, pre-distorted grid, FP64, mimetic current),
timed whole with CUDA events, L2 flushed between steps.  Metric: interior
node-stage updates per second (6 per interior node per attempt).  The block
of K timed attempts is repeated until at least a second of device time has
been timed (so that the clock sampler sees the load); `value` and
`ms_per_step` are the mean over every timed attempt.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one rank per GPU): every rank relaxes its own copy of the
workload (replicas: no data crosses between GPUs) and
`value` is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import glemur_inputs as gi  # noqa: E402

METRIC = "node-stage updates/s"
UNIT = "node-stage/s"
# bytes moved per interior node-stage by the fused layout (stage s reads x,
# B0 and k_1..k_{s-1}, writes k_s; the last writes x_new): 33 fields x 3
# components per accepted step / 6 stages
ALGO_BYTES = {"fp64": 132.0, "mixed": 66.0}
# FP64 flops per interior node-stage of the mimetic stage kernel (FMA = 2),
# counted once per node (halo recomputation excluded)
ALGO_FLOPS_F64 = {"mimetic": 151.0, "direct": 330.0, "nnn": 729.0}
FP64_PEAK_FLOPS = 1.25e12      # nominal dense FP64 rate of GB300 (152 SMs)
L2_FLUSH_BYTES = 512 << 20
MIN_TIMED_S = 1.0              # repeat the block of timed attempts until this
# DRAM bytes per stage from ncu (dram__bytes_read.sum + dram__bytes_write.sum
# of one attempt's six stages, averaged; FP64: both passes of a stage), keyed
# by (workload, precision, curl), with the hash of the kernel sources they were
# captured from (kernel_source_hash()); a workload without an entry, or one
# whose kernels have changed since, reports null
NCU_TRAFFIC = {
    ("braid64", "fp64", "mimetic"): (58517077, "12ef320afb68"),
    ("braid64", "fp64", "direct"): (31328939, "12ef320afb68"),
    ("braid64", "fp64", "nnn"): (44177536, "12ef320afb68"),
    ("periodic64", "fp64", "mimetic"): (58309376, "12ef320afb68"),
    ("braid64", "mixed", "mimetic"): (15706752, "12ef320afb68"),
    ("braid64", "mixed", "direct"): (15828949, "12ef320afb68"),
    ("braid128", "mixed", "mimetic"): (152739371, "12ef320afb68"),
    ("prod384", "mixed", "mimetic"): (4827807787, "12ef320afb68"),
}


# sources the stage kernels and their launches are built from (the adjoint,
# the diagnostics and the allocation-free energy are not on the timed path)
STAGE_SOURCES_EXCLUDED = ("adjoint.cu", "diagnostics.cu", "energy_static.cu")


def kernel_source_hash():
    """First 12 hex digits of the SHA-256 of the stage kernels' CUDA sources
    (sorted by name): the traffic figures above are valid only for the
    kernels they were measured on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1405_0942_gb300", "csrc")
    for p in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))):
        if os.path.basename(p) in STAGE_SOURCES_EXCLUDED:
            continue
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(name, precision, curl):
    ent = NCU_TRAFFIC.get((name, precision, curl))
    if ent is None or ent[1] != kernel_source_hash():
        return None
    return ent[0]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(seconds, units, world, device):
    """Whole-job timing over torch.distributed ranks: the slowest rank's
    time and the units of all ranks (each rank relaxes its own replica)."""
    if world == 1:
        return float(seconds), int(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(u.item()))


# z-periodic counterpart of the 64^3 braid: 64 x 64 nodes across, 62 inner
# planes between the two ghost planes (the same 238,328 interior nodes)
PERIODIC_WORKLOADS = {"periodic64": 64}


def workload(name, n=None):
    if name in PERIODIC_WORKLOADS:
        m = n or PERIODIC_WORKLOADS[name]
        g, x0, B0 = gi.periodic_case(m, m, m - 2, h_z=2.0 / (m - 1))
        return types.SimpleNamespace(grid=g, x0=x0, B0=B0)
    base, nn, _ = gi.WORKLOADS[name]
    return gi.make_workload(base, n=n or nn)


def curl_const(G, curl):
    return {"mimetic": G.MIMETIC, "direct": G.DIRECT, "nnn": G.NNN}[curl]


def new_relaxation(G, w, precision, curl):
    g = w.grid
    return G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi,
                        precision=G.MIXED if precision == "mixed" else G.FP64,
                        curl=curl_const(G, curl), periodic_z=1 if g.periodic_z else 0)


def config_dict(args, w):
    g = w.grid
    if args.workload.startswith("braid"):
        fields = "braid of twist regions on a seeded pre-distorted grid"
    elif args.workload in PERIODIC_WORKLOADS:
        fields = ("two z-periodic twist regions on e_z, periodically pre-distorted grid, "
                  "periodic z boundaries (ghost planes one period from their partners)")
    else:
        fields = args.workload
    return {"workload": args.workload, "grid": [g.nx, g.ny, g.nz],
            "interior_nodes": g.n_interior, "precision": args.precision, "curl": args.curl,
            "fields": fields,
            "step": "one Cash-Karp attempt (6 stages + update/error + control)",
            "l2": "flushed between timed steps (512 MiB write)",
            "lambda0": 1e-7}


# ------------------------------------------------------------------ oracle


def run_oracle_sample(w, max_seconds, max_steps, curl):
    """The FP64 CPU oracle as it stands, one Cash-Karp attempt per step on
    the same workload, bounded in wall time."""
    import oracle as ora
    g = w.grid
    x = w.x0.copy()
    c = {"mimetic": ora.MIMETIC, "direct": ora.DIRECT, "nnn": ora.NNN}[curl]
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        x, lam, rc = ora.step_fixed(g, x, w.B0, 1e-4, c)
        steps += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": g.n_interior * 6 * steps / dt, "unit": UNIT, "cores": 1,
            "kind": "oracle", "seconds": dt, "steps": steps,
            "sample": f"{steps} full FP64 Cash-Karp attempts of the oracle on the "
                      f"{g.nx}x{g.ny}x{g.nz} workload, single thread"}


def _oracle_worker(job):
    """One host core's share of the all-core oracle sample (spawned process)."""
    name, max_seconds, curl = job
    return run_oracle_sample(workload(name), max_seconds, 10 ** 9, curl)


def run_oracle_all_cores(name, max_seconds, curl):
    """The oracle as it stands on every host core: one independent process per
    core, each relaxing its own copy of the workload for `max_seconds`; the
    throughput is the sum.  Processes are spawned (never forked from a
    process that has used the GPU)."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(name, max_seconds, curl)] * n)
    value = sum(r["value"] for r in res)
    steps = sum(r["steps"] for r in res)
    w = workload(name)
    g = w.grid
    return {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
            "seconds": max(r["seconds"] for r in res), "steps": steps,
            "single_core_value": res[0]["value"],
            "sample": f"{steps} full FP64 Cash-Karp attempts of the oracle on the "
                      f"{g.nx}x{g.ny}x{g.nz} workload, {n} independent single-thread "
                      f"processes (one per host core), about {max_seconds:.0f} s each"}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.workload)
    # each core relaxes its own copy for a bounded time: about 4 s per timed
    # step requested, at most 120 s
    cb = run_oracle_all_cores(args.workload, min(120.0, 4.0 * max(args.steps, 1)), args.curl)
    out = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "oracle_attempts": cb["steps"],
           "ms_per_step": 1e3 * w.grid.n_interior * 6 / cb["value"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference", "config": config_dict(args, w), "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ ours


def time_mode(G, torch, w, precision, curl, steps, warmup, flush, min_s=MIN_TIMED_S):
    """CUDA-event times (ms) of blocks of `steps` attempts, each attempt
    timed whole (the target reset and the attempt's kernels, which run back
    to back as programmatic dependents), the block repeated until `min_s`
    seconds of device time have been timed.  Then the per-kernel split (ms,
    launch order: six stages and the step control) of `steps` more attempts
    with an event between stages; those events keep each stage from starting
    early, so the split adds up to a little more than the whole attempt."""
    r = new_relaxation(G, w, precision, curl)
    r.set_x(torch.from_numpy(w.x0).cuda())
    r.set_B0(torch.from_numpy(w.B0).cuda())
    for _ in range(warmup):
        flush.zero_()
        r.attempts(1)
    times = []
    while True:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()                 # L2 flush, outside the event interval
            a.record()
            r.attempts(1)
            b.record()
        torch.cuda.synchronize()
        times.extend(a.elapsed_time(b) for a, b in ev)
        if sum(times) * 1e-3 >= min_s:
            break
    whole = np.array(times)
    split = []
    for _ in range(steps):
        flush.zero_()
        split.append(r.profile_attempt())
    st = r.stats()
    return r, whole, np.array(split), st


FP64_CONTEXT = {}


def fp64_context(torch):
    """Beside the nominal FP64 rate: the SM count of this device and the rate
    cuBLAS's FP64 GEMM reaches on it (4096^3, best of 3 after a warm-up),
    a measured FP64 ceiling for context."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    n = 4096
    a = torch.rand(n, n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    FP64_CONTEXT.update(sm_count=props.multi_processor_count,
                        dgemm_tflops=2.0 * n ** 3 / (best * 1e-3) / 1e12)


def roofline_entry(whole, split, w, name, precision, curl, hbm_peak, peak_kind):
    """Roofline of the stage launches.  Duration basis: the whole timed
    attempt (six stage launches, the step control and the target reset), so
    the achieved rate is a lower bound for the stages themselves; the
    event-separated split gives each stage's share."""
    att_ms = whole.mean()
    I = w.grid.n_interior
    bytes_per_attempt = ALGO_BYTES[precision] * I * 6
    gbs = bytes_per_attempt / (att_ms * 1e-3) / 1e9
    traffic = ncu_traffic(name, precision, curl)
    shares = (split[:, :6].mean(axis=0) / split.sum(axis=1).mean()).round(4).tolist()
    hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
           "frac": gbs / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
           "algorithmic_bytes_per_launch": bytes_per_attempt / 6,
           "duration_basis": "whole attempt / 6 stage launches (CUDA events)",
           "stage_shares": shares}
    if precision == "fp64":
        fl = ALGO_FLOPS_F64[curl] * I * 6 / (att_ms * 1e-3) / 1e12
        alu = {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_FLOPS / 1e12,
               "unit": "TFLOP/s", "frac": fl * 1e12 / FP64_PEAK_FLOPS, "traffic": traffic,
               "peak_kind": "nominal FP64 rate (152 SMs x 2 DFMA/clk x 2.07 GHz)",
               "sm_count": FP64_CONTEXT.get("sm_count"),
               "fp64_dgemm_tflops": FP64_CONTEXT.get("dgemm_tflops"),
               "algorithmic_flops_per_launch": ALGO_FLOPS_F64[curl] * I,
               "duration_basis": hbm["duration_basis"], "stage_shares": shares,
               "hbm_frac": hbm["frac"], "hbm_achieved_gbs": gbs}
        return alu
    return hbm


# bytes per interior node-stage a fused FP64 stage VJP must move: read the
# stage input, B0 and the adjoint of k_s, write the adjoint of the stage
# input, read and write the B0 adjoint (6 FP64 vectors)
ADJ_ALGO_BYTES = 6 * 24.0
# FP64 flops per interior node-stage of the reverse step (FMA = 2): the
# stage recompute 151, the reverse of u = J x B and of the current with the
# current formed again 203, the pull-back reverse with the gathered B
# adjoint 137, the stage-input adjoint gather 18, the reverse Runge-Kutta
# combine 18 (3 + 6 s over the stages' s = 0..5, averaged)
ADJ_ALGO_FLOPS = 527.0


def adjoint_measure(G, torch, w, precision, steps, flush, hbm_peak, peak_kind):
    """One reverse step of the relaxation (glemur_vjp_step: recompute of the
    six stages at x_n, the reverse Runge-Kutta combine and six stage VJPs)
    per timed iteration, CUDA events on the library's stream, L2 flushed
    between iterations."""
    g = w.grid
    r = G.Relaxation(g.nx, g.ny, g.nz, g.lo, g.hi,
                     precision=G.MIXED if precision == "mixed" else G.FP64)
    r.set_x(torch.from_numpy(w.x0).cuda())
    r.set_B0(torch.from_numpy(w.B0).cuda())
    gen = torch.Generator(device="cuda").manual_seed(7)
    lam_next = torch.randn((3, g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda",
                           generator=gen)
    lam = torch.empty_like(lam_next)
    mu = torch.zeros_like(lam_next)
    dt = 1e-3
    for _ in range(2):
        r.vjp_step(dt, lam_next, lam, mu)
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(r.stream)
        r.vjp_step(dt, lam_next, lam, mu)
        e1.record(r.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    I = g.n_interior
    gbs = ADJ_ALGO_BYTES * I * 6 / (ms * 1e-3) / 1e9
    tf = ADJ_ALGO_FLOPS * I * 6 / (ms * 1e-3) / 1e12
    # the reverse kernels run FP64 arithmetic on either storage precision:
    # bound by the FP64 pipe, like the forward FP64 passes
    return {"value": I * 6 / (ms * 1e-3), "unit": "node-stage VJPs/s", "ms_per_step": ms,
            "precision": precision,
            "step": "glemur_vjp_step: six-stage recompute + reverse combine + six stage VJPs",
            "roofline": {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_FLOPS / 1e12,
                         "unit": "TFLOP/s", "frac": tf * 1e12 / FP64_PEAK_FLOPS,
                         "peak_kind": "nominal FP64 rate (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                         "algorithmic_flops_per_node_stage": ADJ_ALGO_FLOPS,
                         "hbm_achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                         "hbm_peak_kind": peak_kind,
                         "algorithmic_bytes_per_node_stage": ADJ_ALGO_BYTES}}


def e2e_measure(G, torch, w, precision, curl, steps):
    """Same step through the C ABI with host buffers: H2D of x and B0 from
    pinned memory, the attempt, D2H of the new positions, per step."""
    r = new_relaxation(G, w, precision, curl)
    xh = torch.from_numpy(w.x0).pin_memory()
    bh = torch.from_numpy(w.B0).pin_memory()
    out = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        r.set_x(xh, non_blocking=True)
        r.set_B0(bh, non_blocking=True)
        r.attempts(1)
        r.get_x(out=out.numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        # pinned inputs copied asynchronously; get_x waits for the result
        r.set_x(xh, non_blocking=True)
        r.set_B0(bh, non_blocking=True)
        r.attempts(1)
        r.get_x(out=out.numpy())
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    nbytes = w.x0.nbytes
    return {"value": w.grid.n_interior * 6 / dt, "unit": UNIT,
            "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": nbytes,
            "ms_per_step": dt * 1e3}


def our_arm(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import paper_1405_0942_gb300 as G
    G.lib()
    hbm_peak, peak_kind = load_peaks()
    w = workload(args.workload)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sampler = ClockSampler(torch.cuda.current_device() if ws == 1 else local)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    if args.precision == "fp64":
        fp64_context(torch)
    barrier()
    sampler.start()
    r, whole, split, st = time_mode(G, torch, w, args.precision, args.curl, args.steps,
                                    args.warmup, flush, args.min_seconds)
    barrier()
    clocks = sampler.stop()
    # device time of every timed attempt; slowest rank, units of all ranks
    total_s, units = reduce_over_ranks(whole.sum() * 1e-3, w.grid.n_interior * 6 * len(whole),
                                       ws, "cuda")
    value = units / total_s
    roof = roofline_entry(whole, split, w, args.workload, args.precision, args.curl, hbm_peak,
                          peak_kind)
    per_kernel = split.mean(axis=0).tolist()

    extra = {}
    if rank == 0 and ws == 1 and not (args.no_compare or args.lean):
        for prec, curl in (("mixed", "mimetic"), ("fp64", "direct"), ("mixed", "direct")):
            if (prec, curl) == (args.precision, args.curl):
                continue
            _, ms2, sp2, st2 = time_mode(G, torch, w, prec, curl, args.steps, args.warmup,
                                         flush, args.min_seconds)
            v2 = w.grid.n_interior * 6 / (ms2.mean() * 1e-3)
            extra[f"{prec}_{curl}"] = {
                "value": v2, "unit": UNIT, "ms_per_step": ms2.mean(),
                "speedup_vs_primary": v2 / value,
                "roofline": roofline_entry(ms2, sp2, w, args.workload, prec, curl, hbm_peak,
                                           peak_kind)}
        if args.workload == "braid64" and args.precision == "fp64":
            # the FP64 two-pass stages with the next-nearest-neighbour
            # current on the same workload, and with periodic z boundaries
            # on its z-periodic counterpart
            for name, curl in (("braid64", "nnn"), ("periodic64", "mimetic")):
                wl = w if name == "braid64" else workload(name)
                _, ms4, sp4, _ = time_mode(G, torch, wl, "fp64", curl, args.steps,
                                           args.warmup, flush, args.min_seconds)
                v4 = wl.grid.n_interior * 6 / (ms4.mean() * 1e-3)
                key = "fp64_nnn" if curl == "nnn" else "fp64_mimetic_periodic64"
                extra[key] = {
                    "value": v4, "unit": UNIT, "ms_per_step": ms4.mean(),
                    "speedup_vs_primary": v4 / value, "workload": name,
                    "grid": [wl.grid.nx, wl.grid.ny, wl.grid.nz],
                    "roofline": roofline_entry(ms4, sp4, wl, name, "fp64", curl, hbm_peak,
                                               peak_kind)}
        if args.workload == "braid64":
            # the mixed-precision path where HBM, not L2, holds the fields:
            # the 128^3 braid of 10 twist regions (mixed-precision workload)
            # and the 384^3 production workload (12 regions + ABC, ~8 GB)
            for name in ("braid128", "prod384"):
                wl = workload(name)
                r3, ms3, sp3, _ = time_mode(G, torch, wl, "mixed", "mimetic", args.steps,
                                            args.warmup, flush, args.min_seconds)
                v3 = wl.grid.n_interior * 6 / (ms3.mean() * 1e-3)
                extra[f"mixed_mimetic_{name}"] = {
                    "value": v3, "unit": UNIT, "ms_per_step": ms3.mean(),
                    "timed_attempts": len(ms3), "workload": name,
                    "grid": [wl.grid.nx, wl.grid.ny, wl.grid.nz],
                    "roofline": roofline_entry(ms3, sp3, wl, name, "mixed", "mimetic", hbm_peak,
                                               peak_kind)}
                del r3, wl
                torch.cuda.empty_cache()
    e2e = None
    if not args.lean:
        # every rank drives its own replica through the C ABI with host
        # buffers; whole-job throughput = units of all ranks / slowest rank
        e2e_steps = max(3, min(args.steps, 10))
        barrier()
        e2e = e2e_measure(G, torch, w, args.precision, args.curl, e2e_steps)
        t_e2e, u_e2e = reduce_over_ranks(e2e["ms_per_step"] * 1e-3 * e2e_steps,
                                         w.grid.n_interior * 6 * e2e_steps, ws, "cuda")
        e2e["value"] = u_e2e / t_e2e
        e2e["ms_per_step"] = t_e2e / e2e_steps * 1e3
        e2e["h2d_bytes_per_step"] *= ws          # all ranks' copies
        e2e["d2h_bytes_per_step"] *= ws
    adj = None
    if rank == 0 and ws == 1 and not args.lean and args.curl == "mimetic":
        adj = adjoint_measure(G, torch, w, args.precision, max(3, min(args.steps, 10)), flush,
                              hbm_peak, peak_kind)
    if ws > 1:
        torch.distributed.barrier()
    if rank != 0:
        return
    cb = (run_oracle_all_cores(args.workload, 12.0, args.curl)
          if ws == 1 and not args.lean else None)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": whole.mean(),
        "timed_attempts": len(whole), "repeats": len(whole) // args.steps,
        "timed_s": float(whole.sum() * 1e-3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded braid field and pre-distorted grid)",
        "config": config_dict(args, w), "roofline": roof, "cpu_baseline": cb, "e2e": e2e,
        "clocks": clocks,
        # the attempts' kernels (the step target is set once, in warm-up)
        "gpu_launches": r.kernels_per_attempt() * len(whole),
        "kernel_ms": {"stages": per_kernel[:6], "control": per_kernel[6]},
        "attempts": {"accepted": st["accepted"], "rejected": st["rejected"]},
        "compare": extra,
        "adjoint": adj,
    }
    print(json.dumps(out), flush=True)


def adjoint_arm(args):
    import torch
    import paper_1405_0942_gb300 as G
    G.lib()
    hbm_peak, peak_kind = load_peaks()
    w = workload(args.workload)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    adj = adjoint_measure(G, torch, w, args.precision, args.steps, flush, hbm_peak, peak_kind)
    out = {"metric": "node-stage VJPs/s", "value": adj["value"], "unit": adj["unit"],
           "n_gpus": 1, "steps": args.steps, "warmup": 2, "ms_per_step": adj["ms_per_step"],
           "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": config_dict(args, w), "roofline": adj["roofline"]}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="braid64",
                    choices=sorted(gi.WORKLOADS) + sorted(PERIODIC_WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--curl", default="mimetic", choices=["mimetic", "direct", "nnn"])
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the reverse step (glemur_vjp_step) and print its line")
    ap.add_argument("--lean", action="store_true",
                    help="timed steps only: no comparisons, e2e or CPU baseline (profiling)")
    ap.add_argument("--min-seconds", type=float, default=MIN_TIMED_S,
                    help="repeat the block of timed steps until this much device time "
                         "(0: time the block once, for profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.adjoint_only:
        adjoint_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
