"""Host logic of the launch planners (csrc/kernels.h), without a GPU.

tests/planner_check.cpp is built with the host C++ compiler against the
library's planner header and run on seeded random batches: every matrix or
front is planned exactly once; each cluster, CTA-group and delayed-update
QRCP launch fits shared memory; CTA groups stay within one CTA per SM and
their exchange areas (arrival counters, slots, reflector buffers) are laid out
back to back with every access range inside its own area; spare CTAs of a group
are spread until each member has at most 8 columns per CTA; FP64 batches put at
most four matrices into CTA groups; front groups respect their size classes.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_launch_planners(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    exe = str(tmp_path / "planner_check")
    src = os.path.join(HERE, "planner_check.cpp")
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I", inc, "-I", os.path.join(ROOT, "paper_2102_09878_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout[-3000:]
