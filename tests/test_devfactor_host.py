"""Host logic of the device decomposition of the W-step operator without a GPU
(Algorithm 2, decompose(L); Sec. 4 "Efficient Evaluation"): tests/devfactor_check.cpp
builds the plan of csrc/ffa_devfactor_plan.cpp for tetrahedral and triangle meshes
(separators of several panels, graded penalties), runs its launch program item by
item on the CPU in double with every access checked against its front, inverse and
block, and compares the blocks with the host multifrontal factor's double blocks;
it also checks the device assembly's term lists against the host assembly of L."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")


def test_device_decomposition_plan_reproduces_the_host_factor(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "devfactor_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-o", exe, os.path.join(ROOT, "tests", "devfactor_check.cpp"),
                    os.path.join(CSRC, "ffa_devfactor_plan.cpp"), os.path.join(CSRC, "ffa_factor.cpp"),
                    os.path.join(CSRC, "ffa_operator_host.cpp")], check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
    # the multi-panel paths ran
    import re
    panels = [int(x) for x in re.findall(r"max panels (\d+)", r.stdout)]
    assert len(panels) == 7 and max(panels) >= 4 and sorted(panels)[-2] >= 3, r.stdout
