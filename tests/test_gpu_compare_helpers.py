"""The FP64 kernels form their compares and min/max of doubles from the bit
patterns (integer ALU) instead of the FP64 unit, and the friction's h^(-1/3)
by Newton's iteration; tests/cuda/compare_helpers_check.cu checks every
comparison helper against the plain IEEE expression it replaces, on special
values (signed zeros, denormals, infinities, NaNs) and seeded random ones, and
the Newton root against CUDA's cbrt.  Built with the package's nvcc for
sm_103a and run on the GPU."""
import os
import subprocess

import pytest

from paper_2010_14416_gb300 import build as libbuild

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2010_14416_gb300", "csrc")


def test_fp64_comparison_helpers_match_ieee(tmp_path):
    exe = str(tmp_path / "compare_helpers_check")
    cmd = [libbuild.nvcc()] + libbuild.ARCH + ["-O3", "-std=c++17", "-I", CSRC,
                                                os.path.join(HERE, "cuda", "compare_helpers_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    counts = dict(line.split() for line in r.stdout.splitlines() if line)
    assert r.returncode == 0, r.stdout + r.stderr
    assert int(counts.pop("values")) > 3000
    ulps = {k: float(counts.pop(k)) for k in ("ulps_r", "ulps_r3", "ulps_r7")}
    assert len(counts) == 11 and all(v == "0" for v in counts.values()), counts
    # the FP64 friction's Newton h^(-1/3) against CUDA's cbrt (relative errors in 2^-52)
    assert ulps["ulps_r"] <= 4 and ulps["ulps_r3"] <= 8 and ulps["ulps_r7"] <= 16, ulps
