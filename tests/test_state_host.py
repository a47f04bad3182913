"""Host logic of ffa_set_state / ffa_get_state without a GPU: tests/state_check.cpp
runs the library's own state packing (csrc/ffa_state.cpp) through the quaternion
convention, round trips of random rotations in 2D and 3D (every branch of
Shepperd's method), the layout of P and Lambda, P's symmetrization and the
refusals of non-rotations and non-finite entries."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")


def test_state_packing_round_trips_and_refusals(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "state_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "state_check.cpp"),
                    os.path.join(CSRC, "ffa_state.cpp")], check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
