"""Host logic of the supernodal-solve schedules, without a GPU: tests/schedule_check.cpp
builds the factor of grid Laplacians with the library's own ffa_factor.cpp, the
task lists and dependency records with ffa_schedule.cpp, and checks tile
coverage, the dynamic lists and the release protocol (replayed sequentially and
by racing threads)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")


def test_schedules_cover_every_block_and_release_every_task_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "schedule_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-o", exe, os.path.join(ROOT, "tests", "schedule_check.cpp"),
                    os.path.join(CSRC, "ffa_factor.cpp"), os.path.join(CSRC, "ffa_schedule.cpp")],
                   check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
