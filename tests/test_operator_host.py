"""Host logic of setup steps a1 and a2 without a GPU: tests/operator_check.cpp runs
the library's own element geometry and operator assembly
(csrc/ffa_operator_host.cpp: hat-function gradients and measures per the
Supplemental "Computing the Jacobian Map"; L = sum_i mu_i G_i^T G_i of eq.
solvinginw restricted to the free vertices, and its device forms) against
affine reproduction, isometric surface triangles, exact measures, L 1 = 0,
symmetry, the quadratic form and the pin block computed element by element, and
the ELL / CSR layouts in elimination order."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")


def test_geometry_assembly_and_device_forms(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "operator_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-o", exe, os.path.join(ROOT, "tests", "operator_check.cpp"),
                    os.path.join(CSRC, "ffa_operator_host.cpp"), os.path.join(CSRC, "ffa_factor.cpp")],
                   check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
