"""ffa_set_state on the GPU (the state of Algorithm 1 between two iterations:
W, U, P, Lambda): the state reads back as set, a run resumed from it continues as
the uninterrupted run does and as the FP64 oracle stepped from the same state,
and the refusals."""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _case(name):
    """The 3D cube, and the 12^2 disk started from the scaled square with its pins
    on the circle (no triangle degenerate to rounding, so neither side's rounding
    decides an orientation)."""
    if name == "cube3d":
        wl = wk.cube_deform(cells=4, seed=93)
        return wl, wl.W0
    wl = wk.uv_disk(grid=12, seed=61, rho=3.0)
    W0 = 1.4 * (wl.V - 0.5)
    W0[wl.pins] = wl.pin_pos
    return wl, W0


@pytest.mark.parametrize("name", ["cube3d", "disk2d"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-5)])
def test_resumed_run_continues_the_uninterrupted_one(name, precision, tol):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl, W0 = _case(name)
    with Solver.from_workload(wl, precision=precision, check_every=5) as a:
        a.init(W0)
        a.iterate(10, stop_at_tol=False)
        W = a.W()
        U, P, L = a.state()
        a.iterate(10, stop_at_tol=False)
        Wa = a.W()
        _, Pa, La = a.state()
    with Solver.from_workload(wl, precision=precision, check_every=5) as b:
        b.set_state(W, U, P, L)
        U2, P2, L2 = b.state()
        # U passes through the quaternion (3D) or (cos, sin) (2D) of the device layout,
        # renormalized on the way in (a float quaternion is unit only to a few ulp)
        assert np.abs(U2 - U).max() <= (1e-13 if precision == "fp64" else 1e-5)
        assert np.array_equal(P2, P) and np.array_equal(L2, L)
        assert np.abs(b.W() - W).max() <= 1e-15 * np.abs(W).max()
        b.iterate(10, stop_at_tol=False)
        Wb = b.W()
        _, Pb, Lb = b.state()
    assert _rel(Wb, Wa) < tol
    assert _rel(Pb, Pa) < 10 * tol
    assert _rel(Lb, La) < 100 * tol


@pytest.mark.parametrize("name", ["cube3d", "disk2d"])
def test_resumed_run_matches_the_oracle_stepped_from_the_same_state(name):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl, W0 = _case(name)
    o = admm.Oracle.from_workload(wl)
    s, _ = o.run(W0, 10, stop_at_tol=False)
    with Solver.from_workload(wl, precision="fp64", check_every=5) as b:
        b.set_state(s.W, s.U, s.P, s.Lam)
        st = b.iterate(10, stop_at_tol=False)
        W = b.W()
        _, P, L = b.state()
    hist = []
    for _ in range(10):
        s, sto = o.step(s)
        hist.append(sto)
    assert _rel(W, s.W) < 1e-8
    assert _rel(P, s.P) < 1e-7
    assert _rel(L, s.Lam) < 1e-6
    assert st["n_flipped"] == hist[-1].n_flipped


def test_refusals():
    _need_gpu()
    from paper_2107_05200_gb300._native import FFAError
    from paper_2107_05200_gb300.solver import Solver
    wl, W0 = _case("cube3d")
    m, d = wl.T.shape[0], 3
    I = np.broadcast_to(np.eye(d), (m, d, d)).copy()
    Z = np.zeros((m, d, d))
    with Solver.from_workload(wl, precision="fp64") as sol:
        with pytest.raises(FFAError, match="not a rotation"):
            sol.set_state(W0, 2.0 * I, I, Z)
        R = I.copy()
        R[5, 2, 2] = -1.0
        with pytest.raises(FFAError, match="not a rotation"):
            sol.set_state(W0, R, I, Z)
        bad = Z.copy()
        bad[3, 0, 1] = np.nan
        with pytest.raises(FFAError, match="non-finite"):
            sol.set_state(W0, I, I, bad)
        # checkpoints of an unrolled forward run are dropped by set_state
        sol.init(W0)
        sol.forward_unrolled(3, 1)
        sol.set_state(W0, I, I, Z)
        with pytest.raises(FFAError, match="has not been called"):
            sol.backward_unrolled(np.zeros_like(W0))
    with Solver.from_workload(wl, penalties="paper") as sol:
        with pytest.raises(FFAError, match="penalty schedule"):
            sol.set_state(W0, I, I, Z)
