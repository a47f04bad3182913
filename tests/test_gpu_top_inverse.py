"""The top levels of the elimination tree solved as x_T = S^-1 t_T between the
triangular passes (top_inverse_levels; Sec. 4, "Efficient Evaluation": the W
step's solve with the fixed factorization of Algorithm 2).

* With the automatic choice and with explicit k, FP64 trajectories equal the
  oracle's at the FP64 parity bound, and the W-step residual stays at double
  rounding level: S^-1 in float acts like the float factor blocks it replaces,
  and the double residual sweeps remove its rounding.
* The same run with and without the top inverse reaches the same W.
* k = n_levels - 1 (only the leaves below T) is still exact; k >= n_levels is
  refused.
* The phase timer reports the product, and the launch count grows by one per
  sweep.
"""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


MESHES = [lambda: wk.cube_deform(cells=10, seed=71),
          lambda: wk.cube_deform(cells=17, seed=72),
          lambda: wk.uv_disk(grid=24, seed=73),
          lambda: wk.uv_heightfield(grid=40, seed=74)]


@pytest.mark.parametrize("k", [-1, 2])
@pytest.mark.parametrize("make", MESHES)
def test_fp64_trajectory_matches_the_oracle(make, k):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    K = 30
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    for _ in range(K):
        s, _ = o.step(s)
    with Solver.from_workload(wl, precision="fp64", check_every=10, top_inverse_levels=k) as sol:
        info = sol.info()
        sol.init(wl.W0)
        sol.iterate(K, stop_at_tol=False)
        W = sol.W()
        res = sol.wstep_residual()
    if k > 0:
        assert info["top_inverse_levels"] == k
    # the automatic choice is off where S^-1's 64 x 64 tiles outweigh the blocks
    # they replace (small separators)
    on = info["top_inverse_levels"] > 0
    assert (info["top_inverse_cols"] > 0) == on and (info["bytes_top_product"] > 0) == on
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert res < 1e-12, res


@pytest.mark.parametrize("make,k_on", [(lambda: wk.cube_deform(cells=17, seed=72), -1),
                                       (lambda: wk.cube_deform(cells=24, seed=77), -1),
                                       (lambda: wk.uv_disk(grid=24, seed=73), 2),
                                       (lambda: wk.uv_heightfield(grid=40, seed=74), 3)])
def test_with_and_without_the_top_inverse(make, k_on):
    """FP32 local step, 20 iterations: the W steps differ only in rounding (the
    automatic choice is on for the 3D cubes)."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    out = {}
    for k in (0, k_on):
        with Solver.from_workload(wl, precision="fp32", check_every=10, top_inverse_levels=k) as sol:
            sol.init(wl.W0)
            sol.iterate(20, stop_at_tol=False)
            out[k] = (sol.W(), sol.wstep_residual(), sol.info())
    W0, r0, i0 = out[0]
    W1, r1, i1 = out[k_on]
    assert i0["top_inverse_levels"] == 0 and i1["top_inverse_levels"] >= 1
    assert i1["bytes_solve_pass"] < i0["bytes_solve_pass"]
    assert r0 < 1e-12 and r1 < 1e-12, (r0, r1)
    assert np.abs(W1 - W0).max() / np.abs(W0).max() < 1e-5


def test_all_but_the_leaves_in_the_top_inverse():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_deform(cells=6, seed=75)
    with Solver.from_workload(wl, precision="fp64", top_inverse_levels=0) as probe:
        levels = probe.info()["n_levels"]
    assert levels >= 3
    K = 20
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    for _ in range(K):
        s, _ = o.step(s)
    with Solver.from_workload(wl, precision="fp64", check_every=10, top_inverse_levels=levels - 1) as sol:
        assert sol.info()["top_inverse_levels"] == levels - 1
        sol.init(wl.W0)
        sol.iterate(K, stop_at_tol=False)
        W = sol.W()
        res = sol.wstep_residual()
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert res < 1e-12, res
    for bad in (levels, 33):
        with pytest.raises(Exception):
            Solver.from_workload(wl, precision="fp64", top_inverse_levels=bad)


def test_phase_times_and_launch_count():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_deform(cells=16, seed=76)
    res = {}
    for k in (0, 2):
        with Solver.from_workload(wl, precision="fp32", check_every=10, top_inverse_levels=k) as sol:
            sol.init(wl.W0)
            sol.iterate(5, stop_at_tol=False)
            res[k] = (sol.profile_phases(5), sol.info())
    (p0, i0), (p2, i2) = res[0], res[2]
    assert p0["ms_top_product"] == 0.0 and p2["ms_top_product"] > 0.0
    assert i2["kernels_per_iteration"] == i0["kernels_per_iteration"] + 2   # two sweeps
    assert i2["setup_seconds_top_inverse"] > 0.0


@pytest.mark.parametrize("factor", ["host", "device"])
@pytest.mark.parametrize("make", [lambda: wk.uv_disk(grid=16, seed=31),
                                  lambda: wk.cube_deform(cells=12, seed=35)])
def test_paper_schedule_recomputes_the_inverse(make, factor):
    """50 iterations of the paper's schedule (6 rescaling events), FP64 local
    step: after each decomposition S^-1 is computed again from the new blocks, so
    the trajectory, penalties and multipliers stay the oracle's."""
    _need_gpu()
    from oracle import schedule
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    K = 50
    o = admm.Oracle.from_workload(wl)
    s, st_o, ne = schedule.run(o, wl.W0, K, stop_at_tol=False)
    with Solver.from_workload(wl, precision="fp64", top_inverse_levels=0) as probe:
        k = min(2, probe.info()["n_levels"] - 1)
    assert k >= 1
    with Solver.from_workload(wl, precision="fp64", penalties="paper", check_every=10, factor=factor,
                              top_inverse_levels=k) as sol:
        assert sol.info()["top_inverse_levels"] == k
        sol.init(wl.W0)
        st = sol.iterate(K, stop_at_tol=False)
        W = sol.W()
        mu = sol.penalties()
        U, P, L = sol.state()
        res = sol.wstep_residual()
    assert st["rescales"] == ne == 6
    np.testing.assert_allclose(mu, o.mu, rtol=1e-8)
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert np.abs(L - s.Lam).max() < 1e-6 * (1.0 + np.abs(s.Lam).max())
    assert res < 1e-12, res


def test_constraints_solve_through_the_inverse():
    """General constraints A W = b: Z = L_FF^-1 A_F^T is formed by solves that run
    through the top product; the FP64 trajectory matches the oracle's KKT solve and
    every iterate is feasible."""
    _need_gpu()
    import scipy.sparse as sp
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_deform(cells=8, seed=47)
    n = wl.V.shape[0]
    pinned = set(int(p) for p in wl.pins)
    free = [v for v in range(n) if v not in pinned]
    rows = np.zeros((2, n))
    rows[0][free[:6]] = 1.0 / 6
    rows[1][free[10]], rows[1][free[-10]] = 1.0, -1.0
    A = sp.csr_matrix(rows)
    b = A @ wl.W0
    K = 20
    o = admm.Oracle.from_workload(wl, constraints=(A, b))
    s, _ = o.run(wl.W0, K, stop_at_tol=False)
    with Solver.from_workload(wl, precision="fp64", check_every=10, top_inverse_levels=2) as sol:
        sol.set_constraints(A, b)
        sol.init(wl.W0)
        sol.iterate(K, stop_at_tol=False)
        W = sol.W()
    np.testing.assert_allclose(A @ W, b, rtol=0, atol=1e-11)
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
