"""The paper's penalty schedule on the GPU (Algorithm 2; Sec. 6, "Rescaling mu_i
and Lambda") against the oracle's schedule (oracle/schedule.py)."""
import numpy as np
import pytest

from oracle import admm, schedule
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle(wl, K):
    o = admm.Oracle.from_workload(wl)
    st_o = {}

    def cb(k, s0, s1, st):
        st_o[k] = st
    s, st, ne = schedule.run(o, wl.W0, K, stop_at_tol=False, callback=cb)
    return o, s, st, ne


@pytest.mark.parametrize("make", [lambda: wk.uv_disk(grid=16, seed=31),
                                  lambda: wk.cube_deform(cells=3, seed=32),
                                  lambda: wk.uv_heightfield(grid=12, seed=33)])
def test_fp64_schedule_matches_the_oracle(make):
    """50 iterations (events after 1..5 and 42): W, mu and Lambda in FP64."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = make()
    K = 50
    o, s, st, ne = _oracle(wl, K)
    with Solver.from_workload(wl, precision="fp64", penalties="paper", check_every=10) as sol:
        sol.init(wl.W0)
        mu0 = sol.penalties()
        st_g = sol.iterate(K, stop_at_tol=False)
        W = sol.W()
        mu = sol.penalties()
        U, P, L = sol.state()
    o0 = admm.Oracle.from_workload(wl)
    s0 = o0.init(wl.W0)
    mu0_o = np.maximum(schedule.mu_min(s0.P, o0.w, wl.energy), o0.w)
    np.testing.assert_allclose(mu0, mu0_o, rtol=1e-10)
    assert st_g["rescales"] == ne == 6
    np.testing.assert_allclose(mu, o.mu, rtol=1e-8)
    assert np.abs(W - s.W).max() / np.abs(s.W).max() < 1e-8
    assert np.abs(L - s.Lam).max() < 1e-6 * (1.0 + np.abs(s.Lam).max())


def test_fp32_schedule_converges_flip_free_on_the_disk():
    """The 48^2 disk: mu = w fixed does not reach the tolerance in 500 iterations;
    the schedule does, with no flipped triangle, in both precisions, at the
    oracle's iteration count to within a few checks."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.uv_disk()
    o = admm.Oracle.from_workload(wl)
    s, st_o, ne = schedule.run(o, wl.W0, 500)
    for prec in ("fp64", "fp32"):
        with Solver.from_workload(wl, precision=prec, penalties="paper", check_every=1) as sol:
            sol.init(wl.W0)
            st = sol.iterate(500, stop_at_tol=True)
        assert st["converged"] == 1 and st["n_flipped"] == 0, (prec, st)
        assert abs(st["iters"] - st_o.k) <= (0 if prec == "fp64" else 20), (prec, st["iters"], st_o.k)


def test_schedule_rejections():
    _need_gpu()
    from paper_2107_05200_gb300._native import FFAError
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_handles(cells=3, seed=34, n_targets=4, lattice_start=1, lattice_step=1)
    with Solver.from_workload(wl, precision="fp64", penalties="paper") as sol:
        sol.init(wl.W0)
        with pytest.raises(FFAError):
            sol.forward_unrolled(4, 2)
    with pytest.raises(ValueError):
        Solver.from_workload(wl, penalties="other")
