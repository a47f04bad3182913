"""Host logic of the top-of-tree inverse, without a GPU: tests/topinv_check.cpp
plans the top levels of grid-Laplacian factors with the library's own
ffa_topinv_plan.cpp, checks the plan against its definition (the supernodes,
their positions and subtree ranges, the structure rows' positions), and emulates
the device setup's steps in double from the float blocks: the result equals the
T block of L_FF^-1 [0; I] from a dense Cholesky factorization, which is S^-1 by
block elimination."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")


def test_top_inverse_plan_and_setup_arithmetic(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "topinv_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-o", exe, os.path.join(ROOT, "tests", "topinv_check.cpp"),
                    os.path.join(CSRC, "ffa_factor.cpp"), os.path.join(CSRC, "ffa_topinv_plan.cpp")],
                   check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
