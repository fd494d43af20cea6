"""Host logic of the multi-SM and CTA-group solve plans, without a GPU.

`tests/plan_check.cpp` is compiled with the host compiler against the planner's source
(`csrc/plan.cpp`) and run.  For several synthetic pose-graph topologies, in both
fill-reducing orderings, it re-derives the symbolic block factorisation by eliminating the
columns in the plan's order and checks against it the planned block rows, the level
schedule (a column above every column that updates it) and the update triplets of every
level.  For cluster sizes 2, 4, 8 and 16 it checks that every update task runs exactly
once per level (near tasks by the owner of their destination), that each CTA's own
triplet list holds exactly the triplets of its tasks in the graph's order, that far tasks
are assigned greedily by estimated work and that the reported shared memory covers every
CTA; and that a batch's CTA-group plan solves every graph once, the slowest on whole
clusters.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2605_30488_b300", "csrc")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        inc = os.path.join(base, "include") if base else ""
        if inc and os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def test_cluster_plan_invariants(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    exe = str(tmp_path / "plan_check")
    cmd = [cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", inc,
           os.path.join(HERE, "plan_check.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
