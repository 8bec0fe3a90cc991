"""Register budget of the single-colony construction kernels, checked at compile time (no GPU).

Three builds of the single-colony construction kernel that compiled to 224-229 registers per
thread raised illegal-address faults on the GPU, each in the code path the build had changed, and
the cause was never found by reading; every build that ran clean compiled to 220-222.  Until that
is understood, a change that takes either stage width's instantiation above 222 registers (or
makes it spill) is not run: this test compiles construct.cu as the library build does and reads
ptxas's report.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1709_03187_gb300", "csrc")
BUDGET = 222


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_single_colony_construction_stays_within_its_register_budget(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    import importlib

    build = importlib.import_module("paper_1709_03187_gb300.build")
    cmd = [nvcc, *build.ARCH, *build.COMMON, "-Xptxas", "-v", "-c", os.path.join(CSRC, "construct.cu"),
           "-o", str(tmp_path / "construct.o")]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    report = {}
    fn = None
    for line in r.stderr.splitlines():
        m = re.search(r"Function properties for (\w+)", line)
        if m:
            fn = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and fn:
            report.setdefault(fn, {})["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and fn:
            report.setdefault(fn, {})["regs"] = int(m.group(1))
            fn = None
    single = {f: v for f, v in report.items() if f.startswith("_Z22construct_lbest_kernelILb0")}
    assert len(single) == 2, report  # the 16- and 24-entry stages
    for f, v in single.items():
        assert v["regs"] <= BUDGET, (f, v)
        assert v.get("spill", 0) == 0, (f, v)
