"""The joint (U, P) prox variant of the local step on the GPU against the
oracle's joint variant (not the paper's scheme; labelled local_variant 1)."""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("make", [lambda: wk.uv_disk(grid=16, seed=51),
                                  lambda: wk.cube_deform(cells=3, seed=52),
                                  lambda: wk.uv_heightfield(grid=12, seed=53)])
def test_fp64_joint_trajectory_matches_the_oracle(make):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    K = 25
    o = admm.Oracle.from_workload(wl, local_variant="joint")
    s = o.init(wl.W0)
    for _ in range(K):
        s, _ = o.step(s)
    with Solver.from_workload(wl, precision="fp64", local_variant="joint", check_every=5) as sol:
        sol.init(wl.W0)
        sol.iterate(K, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert np.abs(P - s.P).max() < 1e-7 * (1.0 + np.abs(s.P).max())
    assert np.abs(L - s.Lam).max() < 1e-6 * (1.0 + np.abs(s.Lam).max())


def test_fp32_joint_converges_where_the_oracle_does():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.uv_disk(grid=24, seed=54)
    o = admm.Oracle.from_workload(wl, local_variant="joint")
    _, st_o = o.run(wl.W0, 500)
    with Solver.from_workload(wl, precision="fp32", local_variant="joint", check_every=1) as sol:
        sol.init(wl.W0)
        st = sol.iterate(500, stop_at_tol=True)
    assert st_o.converged and st["converged"] == 1 and st["n_flipped"] == 0
    assert abs(st["iters"] - st_o.k) <= 5
