"""The numeric decomposition of L_FF on the device (factor_device; Algorithm 2,
decompose(L)) against the host's multifrontal factor and the oracle.

* In double (factor="device64") the float blocks the W step reads equal the host's
  float blocks to one unit in the last place: both round the same double values,
  computed in different orders (agreeing to ~1e-13), to float.
* In float (factor="device") the blocks carry the rounding of a float elimination;
  the W step's double residual sweeps make the solution independent of that, so
  trajectories are compared with the oracle at the FP64 tolerance of the other
  parity tests, and the W-step residual must stay at double rounding level.
* With the paper's penalty schedule every rescaling event assembles L and decomposes
  it on the device; the trajectories, penalties and multipliers match the oracle's
  schedule as with the host decomposition.
* The Tutte initializer with the device decomposition matches the oracle.
"""
import numpy as np
import pytest

from oracle import admm, schedule
from oracle import tutte as ot
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu

ULP32 = 2.0 ** -23


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


MESHES = [lambda: wk.cube_deform(cells=10, seed=51),
          lambda: wk.cube_deform(cells=17, seed=52),       # top separator 18^2 - pins: 5 panels
          lambda: wk.uv_disk(grid=24, seed=53),
          lambda: wk.uv_heightfield(grid=40, seed=54)]


@pytest.mark.parametrize("make", MESHES)
def test_double_device_blocks_equal_the_host_blocks(make):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    with Solver.from_workload(wl, precision="fp64") as h:
        Bh = h.factor_blocks()
        ih = h.info()
    with Solver.from_workload(wl, precision="fp64", factor="device64") as g:
        Bg = g.factor_blocks()
        ig = g.info()
    assert Bh.shape == Bg.shape and ih["factor_entries"] == ig["factor_entries"]
    assert np.all(np.isfinite(Bg))
    scale = np.abs(Bh).max()
    diff = np.abs(Bg.astype(np.float64) - Bh.astype(np.float64))
    bound = ULP32 * np.maximum(np.abs(Bh), np.abs(Bg)).astype(np.float64) + 1e-30 * scale
    assert np.all(diff <= bound), (wl.name, float((diff / np.maximum(np.abs(Bh), 1e-30)).max()))
    # padding and the zeros above the diagonal of inv(L_ss) are exact zeros on both
    np.testing.assert_array_equal(Bg == 0, Bh == 0)


@pytest.mark.parametrize("make", MESHES[:3])
def test_float_device_decomposition_keeps_the_fp64_trajectory(make):
    """FP64 local step, 30 iterations: W with the float device decomposition equals
    the oracle's to 1e-8 (the FP64 parity bound), the W-step residual stays at
    double rounding level, and the blocks are within float elimination error of
    the host's."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    K = 30
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    for _ in range(K):
        s, _ = o.step(s)
    with Solver.from_workload(wl, precision="fp64") as h:
        Bh = h.factor_blocks().astype(np.float64)
    with Solver.from_workload(wl, precision="fp64", factor="device", check_every=10) as g:
        Bg = g.factor_blocks().astype(np.float64)
        g.init(wl.W0)
        g.iterate(K, stop_at_tol=False)
        W = g.W()
        res = g.wstep_residual()
    rel_blocks = np.abs(Bg - Bh).max() / np.abs(Bh).max()
    assert rel_blocks < 1e-3, rel_blocks
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert res < 1e-12, res


@pytest.mark.parametrize("factor", ["device", "device64"])
@pytest.mark.parametrize("make", [lambda: wk.uv_disk(grid=16, seed=31),
                                  lambda: wk.cube_deform(cells=3, seed=32),
                                  lambda: wk.uv_heightfield(grid=12, seed=33),
                                  lambda: wk.cube_deform(cells=12, seed=35)])
def test_schedule_with_device_rescaling_matches_the_oracle(make, factor):
    """50 iterations of the paper's schedule (6 events), FP64 local step: each
    event assembles L from the new penalties and decomposes it on the device."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    K = 50
    o = admm.Oracle.from_workload(wl)
    s, st_o, ne = schedule.run(o, wl.W0, K, stop_at_tol=False)
    with Solver.from_workload(wl, precision="fp64", penalties="paper", check_every=10, factor=factor) as sol:
        sol.init(wl.W0)
        st = sol.iterate(K, stop_at_tol=False)
        W = sol.W()
        mu = sol.penalties()
        U, P, L = sol.state()
        info = sol.info()
    assert st["rescales"] == ne == 6
    np.testing.assert_allclose(mu, o.mu, rtol=1e-8)
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert np.abs(L - s.Lam).max() < 1e-6 * (1.0 + np.abs(s.Lam).max())
    assert info["seconds_refactor"] > 0


def test_device_rescaling_is_faster_than_the_host_on_a_cube():
    """The 24^3 cube under the paper's schedule, 12 iterations (events after 1..5):
    the device assembles and decomposes L at each event; both runs reach the same
    state, the device in less time."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_deform(cells=24, seed=36)
    out = {}
    for factor in ("host", "device"):
        with Solver.from_workload(wl, precision="fp64", penalties="paper", check_every=10, factor=factor) as sol:
            sol.init(wl.W0)
            st = sol.iterate(12, stop_at_tol=False)
            out[factor] = (sol.W(), sol.info()["seconds_refactor"], st["rescales"])
    Wh, th, nh = out["host"]
    Wd, td, nd = out["device"]
    assert nh == nd == 5
    assert np.abs(Wd - Wh).max() / np.abs(Wh).max() < 1e-8
    assert td < th, (td, th)


def test_tutte_with_the_device_decomposition():
    _need_gpu()
    from paper_2107_05200_gb300.solver import tutte
    cube = wk.cube_deform(cells=12, seed=43)
    Wo = ot.tutte(cube.V, cube.T, cube.pins, cube.pin_pos)
    for factor in ("device", "device64"):
        W, rel = tutte(cube.V, cube.T, cube.pins, cube.pin_pos, factor=factor)
        assert rel < 1e-12 and np.abs(W - Wo).max() / np.abs(Wo).max() < 1e-10, factor
    wl = wk.uv_disk(grid=48, seed=41, target_flip=None, sigma=0.0)
    W, rel = tutte(wl.V, wl.T, wl.pins, wl.pin_pos, factor="device")
    assert rel < 1e-12 and np.abs(W - ot.tutte(wl.V, wl.T, wl.pins, wl.pin_pos)).max() < 1e-10


def test_factor_copy_rejects_a_wrong_count():
    _need_gpu()
    import ctypes as C
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_deform(cells=3, seed=32)
    with Solver.from_workload(wl, factor="device") as sol:
        n = sol.info()["factor_entries"]
        buf = np.empty(n + 1, np.float32)
        assert sol._lib.ffa_copy_factor(sol._ctx, buf.ctypes.data, C.c_int64(n + 1)) == 1
        assert sol._lib.ffa_copy_factor(sol._ctx, buf.ctypes.data, C.c_int64(n)) == 0
