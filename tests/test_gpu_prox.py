"""The proximal U term h_i > 0 on the GPU (eq. proximalfunctionu; prox_h = 1) against the
oracle's U step with the same h_i: h_i = 4 w_i^2 B_i^2 / mu_i at the bound of Prop. 1,
B_i = sqrt(5 (1 + |grad f(P_i^0)|^2)) with gamma = 1, eps = 0 (Sec. 6), the oracle's
weight coming from oracle.schedule.h_bound on the oracle's own P^0."""
import numpy as np
import pytest

from oracle import admm, schedule
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _solver(wl, **kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05200_gb300.solver import Solver
    return Solver.from_workload(wl, **kw)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _cases():
    return {
        # unflipped starts: the case Sec. 6 turns the proximal term on for
        "disk_sd_unflipped": wk.uv_disk(grid=14, seed=51, target_flip=None, sigma=0.002, rho=3.0),
        "cube_sd_unflipped": wk.cube_deform(cells=4, seed=52, angle_deg=10.0, shift_x=0.05),
        "surface_sg": wk.uv_heightfield(grid=16, seed=53),
        "cube_sa": wk.cube_deform(cells=3, seed=54, energy="sa"),
    }


def _oracle_prox_run(wl, iters):
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    o.h = schedule.h_bound(s.P, o.w, o.mu, wl.energy)
    hist = []
    for _ in range(iters):
        s, st = o.step(s)
        hist.append(st)
    return o, s, hist


@pytest.mark.parametrize("name", ["disk_sd_unflipped", "cube_sd_unflipped", "surface_sg", "cube_sa"])
def test_fp64_trajectory_with_proximal_u_term(name):
    wl = _cases()[name]
    iters = 20
    o, s, hist = _oracle_prox_run(wl, iters)
    assert np.all(o.h > 0)
    with _solver(wl, precision="fp64", check_every=5, prox_h=True) as sol:
        sol.init(wl.W0)
        st = sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    assert _rel(W, s.W) < 1e-8
    assert _rel(U, s.U) < 1e-7
    assert _rel(P, s.P) < 1e-7
    assert _rel(L, s.Lam) < 1e-6
    assert st["n_flipped"] == hist[-1].n_flipped
    # the term matters: the run without it ends elsewhere
    with _solver(wl, precision="fp64", check_every=5) as sol0:
        sol0.init(wl.W0)
        sol0.iterate(iters, stop_at_tol=False)
        assert _rel(sol0.W(), s.W) > 1e-6


@pytest.mark.parametrize("name", ["disk_sd_unflipped", "cube_sd_unflipped"])
def test_fp32_with_proximal_u_term_within_tolerance(name):
    wl = _cases()[name]
    iters = 20
    o, s, hist = _oracle_prox_run(wl, iters)
    with _solver(wl, precision="fp32", check_every=5, prox_h=True) as sol:
        sol.init(wl.W0)
        sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
    assert _rel(W, s.W) < 1e-5


def test_proximal_term_refusals():
    from paper_2107_05200_gb300._native import FFAError
    wl = wk.uv_disk(grid=6)
    with pytest.raises(FFAError, match="INVALID_ARG"):
        _solver(wl, prox_h=True, penalties="paper")
    with pytest.raises(FFAError, match="INVALID_ARG"):
        _solver(wl, prox_h=True, local_variant="joint")
    with _solver(wl, prox_h=True) as sol:
        sol.init(wl.W0)
        with pytest.raises(FFAError, match="INVALID_ARG"):
            sol.forward_unrolled(4, 2)
