"""Host logic of ffa_set_constraints without a GPU: tests/constraint_check.cpp runs
the library's own split of A into free and pinned parts and its Schur-complement
inverse (csrc/ffa_constraint_host.cpp), and checks on dense random problems that
the projection X0 - Z S^-1 (A_F X0 - b') applied on the GPU equals the KKT
solution of Sec. 4's constrained W step."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")


def test_split_schur_inverse_and_projection(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "constraint_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "constraint_check.cpp"),
                    os.path.join(CSRC, "ffa_constraint_host.cpp")], check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
