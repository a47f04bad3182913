"""The benchmark's command-line contract on a machine without a GPU: the oracle
arm (`--impl reference`, the plain FP64 CPU restatement timed on the host) prints
one JSON line with the keys the contract names, and the GPU arm refuses to run
instead of falling back to the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def _run(args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "0", "--cpu-sample-cells", "6",
              "--growth-cells", "8", "10"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference"
    assert out["value"] > 0 and out["ms_per_step"] > 0
    assert out["steps"] == 2 and out["warmup"] == 0 and out["n_gpus"] == 1
    assert out["higher_is_better"] is True
    # the config names the mesh the oracle actually ran; the extrapolation is separate
    assert out["config"]["workload"] == "cube_deform_6" and out["config"]["tets"] == 6 * 6 ** 3
    ext = out["extrapolated_to"]
    assert ext["workload"] == "cube_deform_64" and ext["tets"] == 6 * 64 ** 3
    assert 0.5 < ext["growth_exponent"] < 2.0 and ext["s_per_iter"] > 0
    assert out["sample_timed"]["iterations"] == 2 and out["sample_timed"]["setup_s"] > 0
    assert all(v["setup_s"] > 0 and v["s_per_iter"] > 0 for v in out["cpu_baseline"]["sizes"].values())
    assert out["cpu_baseline_all_threads"]["cores"] >= 1
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == out["value"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.skipif(_cuda_available(), reason="a CUDA device is present")
def test_gpu_arm_refuses_without_a_device():
    r = _run(["--steps", "1", "--warmup", "0"])
    assert r.returncode != 0
    assert "CUDA" in (r.stdout + r.stderr)
    assert not any(ln.strip().startswith("{") for ln in r.stdout.splitlines())


def test_oracle_extrapolation_rule():
    """bench.extrapolate: the largest sample scaled by the element-count ratio to the
    power measured between the two largest samples (medians), linear with one sample."""
    import math
    sys.path.insert(0, ROOT)
    import bench
    m_full = 1_572_864
    # an exact power law is reproduced exactly, whatever the smaller samples do
    samples = {16: (24_576, [9.0, 0.1, 0.2], 0.1), 24: (82_944, [2.0 * 82_944 ** 1.1] * 3, 0.1),
               32: (196_608, [2.0 * 196_608 ** 1.1] * 5, 0.1)}
    t, a = bench.extrapolate(samples, m_full)
    assert math.isclose(a, 1.1, rel_tol=1e-12) and math.isclose(t, 2.0 * m_full ** 1.1, rel_tol=1e-12)
    # the median of each size's iterations is used
    samples[32] = (196_608, [2.0 * 196_608 ** 1.1, 1e9, 0.0, 2.0 * 196_608 ** 1.1, 1.0], 0.1)
    assert math.isclose(bench.extrapolate(samples, m_full)[1], 1.1, rel_tol=1e-12)
    # one sample: linear in the element count
    t1, a1 = bench.extrapolate({16: (24_576, [0.25, 0.3, 0.2], 0.1)}, m_full)
    assert a1 == 1.0 and math.isclose(t1, 0.25 * m_full / 24_576, rel_tol=1e-12)
