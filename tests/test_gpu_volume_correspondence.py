"""The volume-correspondence workload on the GPU (Sec. Results, "Volume
Correspondence") against the oracle: the Tutte start computed by ffa_tutte equals
the workload's, the FP64 trajectory from it matches the oracle's, and the FP32 run
reaches the termination test with no flipped tetrahedron although the start has
some."""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("cells", [8, 20])
def test_gpu_tutte_start_equals_the_workloads(cells):
    _need_gpu()
    from paper_2107_05200_gb300.solver import tutte
    wl = wk.volume_correspondence(cells=cells)
    for factor in ("host", "device"):
        W, rel = tutte(wl.V, wl.T, wl.pins, wl.pin_pos, factor=factor)
        assert rel < 1e-12
        assert np.abs(W - wl.W0).max() / np.abs(wl.W0).max() < 1e-10, factor


def test_fp64_trajectory_matches_the_oracle():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.volume_correspondence(cells=8)
    assert wl.meta["flipped0"] > 0.0
    K = 30
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    for _ in range(K):
        s, _ = o.step(s)
    with Solver.from_workload(wl, precision="fp64", check_every=10) as sol:
        sol.init(wl.W0)
        sol.iterate(K, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert np.abs(L - s.Lam).max() < 1e-6 * (1.0 + np.abs(s.Lam).max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_runs_to_a_flip_free_correspondence(precision):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.volume_correspondence(cells=8)
    o = admm.Oracle.from_workload(wl)
    _, st_o = o.run(wl.W0, 400, stop_at_tol=True)
    assert st_o.converged
    with Solver.from_workload(wl, precision=precision, check_every=1) as sol:
        sol.init(wl.W0)
        st = sol.iterate(400, stop_at_tol=True)
    assert st["converged"] == 1 and st["n_flipped"] == 0, st
    assert abs(st["iters"] - st_o.k) <= (0 if precision == "fp64" else 10), (st["iters"], st_o.k)
