"""Host planner invariants (no GPU): tests/plan/plan_check.cpp is compiled
against csrc/sm_plan.h with the host compiler and run on random patterns.
It checks that every plan lists each compare once, that the window groups
the kernels read describe exactly the peeled compares (window, word class,
shift), and that the symbol bits chosen for 1-bit and 2-bit codes separate
the text's symbols."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "plan", "plan_check.cpp")
CSRC = os.path.join(ROOT, "paper_1612_01506_gb300", "csrc")


@pytest.fixture(scope="module")
def plan_check(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, SRC, "-o", exe])
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_planner_invariants(plan_check, seed):
    out = subprocess.run([plan_check, str(seed), "5000"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
