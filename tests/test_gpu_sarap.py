"""The symmetric ARAP energy (FFA_SYM_ARAP) on the GPU against the FP64 oracle:
trajectories of the local step in both precisions, the energy and its gradient,
a batch mixing all three energies, the adjoint against central differences of
the oracle, and the refusal of the penalty schedule (Lemma 1 covers SD and SG)."""
import math

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


def _oracle_run(wl, iters):
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    hist = []
    for _ in range(iters):
        s, st = o.step(s)
        hist.append(st)
    return o, s, hist


def _workloads():
    return {
        "disk2d": wk.uv_disk(grid=14, seed=91, rho=3.0, energy="sa"),
        "surface": wk.uv_heightfield(grid=16, seed=92, energy="sa"),
        "cube3d": wk.cube_deform(cells=4, seed=93, energy="sa"),
    }


@pytest.mark.parametrize("name", ["disk2d", "surface", "cube3d"])
def test_fp64_trajectory_matches_the_oracle(name):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = _workloads()[name]
    iters = 25
    o, s, hist = _oracle_run(wl, iters)
    with Solver.from_workload(wl, precision="fp64", check_every=5) as sol:
        sol.init(wl.W0)
        st = sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    assert _rel(W, s.W) < 1e-8
    assert _rel(P, s.P) < 1e-7
    assert _rel(L, s.Lam) < 1e-6
    ref = hist[-1]
    assert math.isclose(st["e_prim"], ref.e_prim, rel_tol=1e-6, abs_tol=1e-12)
    assert math.isclose(st["energy_P"], ref.energy_P, rel_tol=1e-9)
    assert st["n_flipped"] == ref.n_flipped


@pytest.mark.parametrize("name", ["disk2d", "cube3d"])
def test_fp32_trajectory_within_stated_tolerance(name):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = _workloads()[name]
    iters = 25
    o, s, hist = _oracle_run(wl, iters)
    with Solver.from_workload(wl, precision="fp32", check_every=5) as sol:
        sol.init(wl.W0)
        st = sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
    assert _rel(W, s.W) < 1e-5
    assert math.isclose(st["energy_P"], hist[-1].energy_P, rel_tol=1e-5)


def test_energy_and_gradient():
    """At a map with moderate distortion (an affine stretch plus noise): FP64 to
    rounding, FP32 within the stated bounds; a flipped map has infinite energy."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_deform(cells=3, seed=94, energy="sa")
    rng = np.random.default_rng(4)
    A = np.array([[1.3, 0.2, 0.0], [0.0, 0.8, 0.1], [0.1, 0.0, 1.1]])
    W = wl.V @ A.T + 0.01 * rng.normal(size=wl.V.shape)
    o = admm.Oracle.from_workload(wl)
    for prec, etol, gtol in (("fp64", 1e-12, 1e-10), ("fp32", 1e-6, 1e-4)):
        with Solver.from_workload(wl, precision=prec) as sol:
            assert math.isclose(sol.energy(W), o.energy(W), rel_tol=etol)
            assert _rel(sol.gradient(W), o.energy_gradient(W)) < gtol
            Wf = W.copy()
            Wf[:, 0] *= -1
            assert sol.energy(Wf) == math.inf


def test_fp32_disk_unflips_and_converges():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.uv_disk(grid=20, seed=73, rho=3.0, energy="sa")
    o = admm.Oracle.from_workload(wl)
    so, sto = o.run(wl.W0, 600)
    with Solver.from_workload(wl, precision="fp32", check_every=10) as sol:
        sol.init(wl.W0)
        st = sol.iterate(600)
        W = sol.W()
    assert st["converged"] == 1 and st["n_flipped"] == 0
    assert wk.flipped_fraction(W, wl.T) == 0.0
    assert abs(st["checked_iter"] - sto.k) <= 10
    assert math.isclose(o.energy(W), o.energy(so.W), rel_tol=1e-4)


def test_batch_mixing_three_energies_matches_single_solves():
    _need_gpu()
    from paper_2107_05200_gb300.solver import BatchSolver, Solver
    wls = [wk.uv_disk(grid=10, seed=95, rho=3.0, energy="sa"),
           wk.uv_disk(grid=12, seed=96, rho=3.0, energy="sd"),
           wk.uv_disk(grid=11, seed=97, rho=3.0, energy="sg")]
    iters = 30
    with BatchSolver(wls, precision="fp64", check_every=10) as bs:
        bs.init([wl.W0 for wl in wls])
        bs.iterate(iters, stop_at_tol=False)
        Wb = [bs.W(j) for j in range(len(wls))]
    for j, wl in enumerate(wls):
        with Solver.from_workload(wl, precision="fp64", check_every=10) as sol:
            sol.init(wl.W0)
            sol.iterate(iters, stop_at_tol=False)
            assert _rel(Wb[j], sol.W()) < 1e-9


def test_adjoint_matches_oracle_central_differences():
    """dL/db of 10 unrolled FP64 iterations on a small handle cube with f_SA against
    central differences (h = 1e-6) of the oracle's loss, for every pin coordinate."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_handles(cells=4, seed=98, n_targets=12, lattice_start=1, lattice_step=2, pre_bend=0.5,
                         energy="sa")
    K = 10
    tgt_idx, tgt = wl.meta["target_idx"], wl.meta["targets"]

    def loss_grad(W):
        r = W[tgt_idx] - tgt
        G = np.zeros_like(W)
        G[tgt_idx] = 2.0 * r / len(tgt_idx)
        return float(np.mean(np.sum(r * r, axis=1))), G

    with Solver.from_workload(wl, precision="fp64") as sol:
        sol.set_handles(wl.pin_pos)
        sol.init(wl.W0)
        sol.forward_unrolled(K, 5)
        _, G = loss_grad(sol.W())
        gb = sol.backward_unrolled(G)

    def oracle_loss(b):
        o = admm.Oracle(wl.V, wl.T, wl.pins, b, wl.energy, wl.rho)
        s, _ = o.run(wl.W0, K, stop_at_tol=False)
        return loss_grad(s.W)[0]

    h = 1e-6
    fd = np.zeros_like(wl.pin_pos)
    for p in range(wl.pin_pos.shape[0]):
        for c in range(wl.pin_pos.shape[1]):
            bp, bm = wl.pin_pos.copy(), wl.pin_pos.copy()
            bp[p, c] += h
            bm[p, c] -= h
            fd[p, c] = (oracle_loss(bp) - oracle_loss(bm)) / (2 * h)
    assert np.linalg.norm(gb - fd) <= 1e-6 * np.linalg.norm(fd)


def test_refusals():
    _need_gpu()
    from paper_2107_05200_gb300._native import FFAError
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.uv_disk(grid=8, seed=99, energy="sa")
    with pytest.raises(FFAError, match="Lemma 1"):
        Solver.from_workload(wl, penalties="paper")
