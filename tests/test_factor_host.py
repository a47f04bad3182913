"""Host logic of the fixed W-step operator's factorization without a GPU:
tests/factor_check.cpp factors SPD matrices with the sparsity of 2D and 3D meshes
and strongly graded weights with the library's own csrc/ffa_factor.cpp (nested
dissection, multifrontal Cholesky, blocks [inv(L_ss); L_rs inv(L_ss)], Sec. 4
"Efficient Evaluation") and checks the permutation and block layout, the
backward error of a solve with the double blocks, the float blocks as the
rounded double ones, bitwise independence of the thread count, refactor against
a fresh factorization, and the refusal of an indefinite matrix."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")


def test_factor_solves_and_is_deterministic(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "factor_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-o", exe, os.path.join(ROOT, "tests", "factor_check.cpp"),
                    os.path.join(CSRC, "ffa_factor.cpp")], check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
