"""The FP64 stages' reciprocal 1/det G (Newton-Raphson refinement of the
hardware approximation) against the IEEE quotient, on 4M log-uniform
inputs: compiled from the library's own header on the GPU machine."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1405_0942_gb300", "csrc")
PROBE = os.path.join(ROOT, "tests", "probes", "recip_probe.cu")


def _nvcc():
    exe = shutil.which("nvcc")
    if exe is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        exe = "/usr/local/cuda/bin/nvcc"
    return exe


def test_fp64_reciprocal_within_an_ulp_of_ieee(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "recip_probe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", CSRC, "-o", exe, PROBE], check=True)
    out = subprocess.run([exe, str(1 << 22), "7"], check=True, capture_output=True,
                         text=True, timeout=120).stdout.split()
    vals = dict(zip(out[0::2], out[1::2]))
    assert int(vals["n"]) == 1 << 22
    # two Newton steps from a 2^-20 approximation: error ~2^-80 before the
    # final rounding, so at most one ulp from the correctly rounded quotient
    assert int(vals["max_ulp"]) <= 1, vals
