"""Task shapes of the supernodal solves: merged bottom subtrees (one block runs a
small subtree's supernodes in order), narrow supernodes cut into row tiles, and
ffa_autotune's choice among them; each under the dynamic schedule (1) and the
pipelined one (2: a producer warp streams the factor into a shared-memory ring).  Every shape must give the same W step: the
iterates are compared with the level-by-level schedule, the FP64 oracle and the
double-precision residual of the refined solve (eq. solvinginw)."""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(wl, iters, **kw):
    from paper_2107_05200_gb300.solver import Solver
    with Solver.from_workload(wl, precision="fp64", check_every=5, **kw) as sol:
        sol.init(wl.W0)
        sol.iterate(iters, stop_at_tol=False)
        return sol.W(), sol.wstep_residual()


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("heights", [(0, 0), (1, 1), (2, 2), (3, 3), (8, 8), (2, 1)])
def test_merged_subtrees_give_the_level_schedule_iterates(heights, schedule):
    """Cube of 20^3 cells (48k tets, 13 tree levels): every merge height, per pass."""
    _need_gpu()
    wl = wk.cube_deform(cells=20, seed=61)
    W_ref, r_ref = _run(wl, 10, schedule=0)
    W, r = _run(wl, 10, schedule=schedule, subtree_height=heights)
    assert r < 1e-12 and r_ref < 1e-12
    np.testing.assert_allclose(W, W_ref, rtol=0, atol=1e-11 * np.abs(W_ref).max())


@pytest.mark.parametrize("schedule", [1, 2])
def test_merged_subtrees_match_the_oracle_on_a_surface_mesh(schedule):
    """2D heightfield of 40^2 vertices with the deepest merge: 15 iterations
    against the FP64 oracle."""
    _need_gpu()
    wl = wk.uv_heightfield(grid=40, seed=62)
    W, r = _run(wl, 15, schedule=schedule, subtree_height=(8, 8))
    o = admm.Oracle.from_workload(wl)
    s, _ = o.run(wl.W0, 15, stop_at_tol=False)
    assert r < 1e-12
    np.testing.assert_allclose(W, s.W, rtol=0, atol=1e-8 * np.abs(s.W).max())


def test_autotune_reports_its_choices_and_keeps_the_iterate():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_deform(cells=16, seed=63)
    with Solver.from_workload(wl, precision="fp64", check_every=5) as a, \
            Solver.from_workload(wl, precision="fp64", check_every=5) as b:
        a.init(wl.W0)
        b.init(wl.W0)
        a.iterate(3, stop_at_tol=False)
        b.iterate(3, stop_at_tol=False)
        t = a.autotune(2)
        assert t["local_block"] in (64, 128, 256) and t["narrow_cols"] in (32, 64)
        assert t["schedule"] in (0, 1, 2) and t["bottom_levels"] in (0, 2, 3, 4)
        assert all(ms > 0 for ms in t["ms_schedule"])
        assert all(0 <= h <= 3 for h in t["subtree_height"])
        if t["schedule"] == 1 and t["bottom_levels"] == 0:
            assert all(ms > 0 for row in t["ms_subtree"] for ms in row)
        a.iterate(7, stop_at_tol=False)
        b.iterate(7, stop_at_tol=False)
        Wa, Wb = a.W(), b.W()
        assert a.wstep_residual() < 1e-12
        np.testing.assert_allclose(Wa, Wb, rtol=0, atol=1e-11 * np.abs(Wb).max())


@pytest.mark.parametrize("cells", [32, 48])
def test_pipelined_schedule_on_larger_cubes(cells):
    """Larger trees (wide tiles cut from supernodes of up to thousands of columns, bands
    above the diagonal skipped): the pipelined passes give the per-level schedule's W."""
    _need_gpu()
    wl = wk.cube_deform(cells=cells, seed=64)
    W_ref, r_ref = _run(wl, 4, schedule=0)
    W, r = _run(wl, 4, schedule=2)
    assert r < 1e-12 and r_ref < 1e-12
    np.testing.assert_allclose(W, W_ref, rtol=0, atol=1e-11 * np.abs(W_ref).max())
