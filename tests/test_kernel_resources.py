"""Register budget of the kernels the tuned benchmarks run: ptxas reports no
local-memory spills for them (a spill in the flux path costs several percent
per step).  Runs nvcc only, no GPU."""
import os
import re
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2010_14416_gb300 import build as libbuild

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2010_14416_gb300", "csrc")
INCLUDE = os.path.join(HERE, "..", "include")

# (translation unit, mangled-name fragment) of the kernels the tuned runs use:
# the 13M river's activity kernel, the fully wet river's step kernels (one
# cell and cell pairs per thread), the FP32
# ensemble's activity kernel with dynamically taken chunks, the FP64 edge pass
# (edge kernel and cell pass) and the FP64 ensemble's cell pass
KERNELS = [
    ("swe_step_f32.cu", "15step_kernel_actIfLi128ELi8ELb1ELi2E"),
    ("swe_step_f32.cu", "11step_kernelIfLi256ELi4ELi3ELb1ELb0E"),
    ("swe_step_f32.cu", "11step_kernelIfLi128ELi8ELi3ELb1ELb0E"),
    ("swe_step_f32.cu", "24ensemble_step_kernel_actIfLi128ELi8ELb1ELb1ELb0E"),
    ("swe_step_f32.cu", "16step_kernel_pairILi256ELi4ELb1EE"),
    ("swe_step_f32.cu", "16step_kernel_pairILi128ELi8ELb1EE"),
    ("swe_step_f32.cu", "25ensemble_step_kernel_pairILi128ELi8ELb1EE"),
    ("swe_step_f32.cu", "24ensemble_step_kernel_actIfLi128ELi7ELb1ELb1ELb1E"),
    ("swe_step_f32.cu", "24ensemble_step_kernel_actIfLi128ELi7ELb1ELb0ELb1E"),
    ("swe_step_f64.cu", "16edge_flux_kernelIdLi256E"),
    ("swe_step_f64.cu", "11step_kernelIdLi128ELi1ELi1ELb0ELb1E"),
    ("swe_step_f64.cu", "20ensemble_step_kernelIdLi128ELi1ELi1ELb0ELb1E"),
]


def _ptxas_report(unit, extra):
    cmd = [libbuild.nvcc()] + libbuild.ARCH + ["-O3", "-std=c++17", "-I", INCLUDE, "-Xptxas", "-v"] + extra + [
        "-c", os.path.join(CSRC, unit), "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    # ptxas prints "Compiling entry function '<name>'" then the function's
    # properties, including "<n> bytes spill stores, <m> bytes spill loads"
    spills, current = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            current = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and current:
            spills[current] = (int(m.group(1)), int(m.group(2)))
            current = None
    return spills


def test_tuned_kernels_do_not_spill():
    try:
        libbuild.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    units = {"swe_step_f32.cu": ["--use_fast_math"], "swe_step_f64.cu": []}
    with ThreadPoolExecutor(max_workers=2) as ex:
        reports = dict(zip(units, ex.map(lambda u: _ptxas_report(u, units[u]), units)))
    for unit, frag in KERNELS:
        found = {name: sp for name, sp in reports[unit].items() if frag in name}
        assert found, f"{frag} not compiled in {unit}"
        for name, sp in found.items():
            assert sp == (0, 0), f"{name}: {sp[0]} bytes spill stores, {sp[1]} bytes spill loads"
