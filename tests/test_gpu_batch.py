"""Batched meshes: every mesh of a batch follows the same iterates as its own
single-mesh solve (and therefore the oracle), with per-mesh statistics and
per-mesh termination."""
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


def _batch_workloads():
    wls = wk.batched_meshes(count=6, seed=7, m_min=300, m_max=3000)
    # a mesh without pins: vertex 0 is fixed at the origin
    nop = wk.uv_disk(grid=10, seed=8, rho=3.0, tol=1e-5)
    nop.pins = np.zeros(0, np.int32)
    nop.pin_pos = np.zeros((0, 2))
    return wls + [nop]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_batch_matches_single_mesh_solves(precision, tol):
    _need_gpu()
    from paper_2107_05200_gb300.solver import BatchSolver, Solver
    wls = _batch_workloads()
    K = 30
    with BatchSolver(wls, precision=precision, check_every=10) as bs:
        bs.init([wl.W0 for wl in wls])
        stats, _ = bs.iterate(K, stop_at_tol=False)
        Wb = [bs.W(j) for j in range(len(wls))]
    for j, wl in enumerate(wls):
        with Solver.from_workload(wl, precision=precision, check_every=10) as sol:
            sol.init(wl.W0)
            st = sol.iterate(K, stop_at_tol=False)
            W = sol.W()
        err = np.abs(Wb[j] - W).max() / np.abs(W).max()
        assert err < tol, (j, err)
        for key in ("e_prim", "e_dual", "thr_prim", "thr_dual", "energy_P"):
            assert math.isclose(stats[j][key], st[key], rel_tol=1e-6 if precision == "fp64" else 1e-2,
                                abs_tol=1e-12), (j, key, stats[j][key], st[key])
        assert stats[j]["n_flipped"] == st["n_flipped"]


@pytest.mark.parametrize("factor", ["device", "device64"])
def test_batch_with_the_device_decomposition_matches_single_mesh_solves(factor):
    """Each group's block-diagonal L_FF decomposed on the device (float or double):
    FP64 local step, every mesh within 1e-9 of its own solve with the host's
    decomposition."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import BatchSolver, Solver
    wls = _batch_workloads()
    K = 20
    with BatchSolver(wls, precision="fp64", check_every=10, factor=factor) as bs:
        bs.init([wl.W0 for wl in wls])
        bs.iterate(K, stop_at_tol=False)
        Wb = [bs.W(j) for j in range(len(wls))]
    for j, wl in enumerate(wls):
        with Solver.from_workload(wl, precision="fp64", check_every=10) as sol:
            sol.init(wl.W0)
            sol.iterate(K, stop_at_tol=False)
            W = sol.W()
        err = np.abs(Wb[j] - W).max() / np.abs(W).max()
        assert err < 1e-9, (factor, j, err)


def test_batch_matches_the_oracle_and_stops_when_all_meshes_converged():
    _need_gpu()
    from paper_2107_05200_gb300.solver import BatchSolver
    wls = wk.batched_meshes(count=4, seed=9, m_min=300, m_max=1500)
    K = 20
    with BatchSolver(wls, precision="fp64", check_every=5) as bs:
        bs.init([wl.W0 for wl in wls])
        bs.iterate(K, stop_at_tol=False)
        Wb = [bs.W(j) for j in range(len(wls))]
        stats, nconv = bs.iterate(2000, stop_at_tol=True)
    for j, wl in enumerate(wls):
        o = admm.Oracle.from_workload(wl)
        s = o.init(wl.W0)
        for _ in range(K):
            s, _ = o.step(s)
        assert np.abs(Wb[j] - s.W).max() / np.abs(s.W).max() < 1e-8, j
    assert nconv == len(wls)
    assert all(st["converged"] == 1 and st["n_flipped"] == 0 for st in stats)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_statistics_repeat_and_tiny_meshes_get_their_own_sums(precision):
    """The per-mesh sums of the termination test are formed in a fixed order (no
    floating-point atomics); tiny meshes (a single element, a few elements) share
    blocks with their neighbours and still get exactly their own sums (checked
    against their single-mesh solves).  Two runs of the same batch agree to
    rounding: the W step's supernodal passes scatter with float atomics, so the
    iterates themselves differ between runs in the last bits."""
    _need_gpu()
    from paper_2107_05200_gb300.solver import BatchSolver, Solver
    wls = wk.batched_meshes(count=5, seed=11, m_min=300, m_max=4000)
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
    tri = wk.Workload("tri", V, np.array([[0, 1, 2]], np.int32), np.array([0], np.int32), V[:1].copy(),
                      V * 1.3 + 0.05, "sd", rho=3.0, eps_abs=1e-5, eps_rel=1e-4)
    small = wk.uv_disk(grid=4, seed=12, rho=3.0, tol=1e-5)
    wls = [wls[0], tri, small, wls[1], tri, wls[2], small, wls[3], wls[4]]
    runs = []
    for _ in range(2):
        with BatchSolver(wls, precision=precision, check_every=5) as bs:
            bs.init([wl.W0 for wl in wls])
            stats, _ = bs.iterate(15, stop_at_tol=False)
            runs.append(stats)
    rtol = 1e-10 if precision == "fp64" else 1e-4
    for a, b in zip(*runs):
        for key in ("e_prim", "e_dual", "thr_prim", "thr_dual", "energy_P", "norm_GtLambda"):
            assert math.isclose(a[key], b[key], rel_tol=rtol, abs_tol=1e-13), (key, a[key], b[key])
    for j in (1, 2):
        with Solver.from_workload(wls[j], precision=precision, check_every=5) as sol:
            sol.init(wls[j].W0)
            st = sol.iterate(15, stop_at_tol=False)
        for key in ("e_prim", "e_dual", "thr_prim", "thr_dual", "energy_P"):
            assert math.isclose(runs[0][j][key], st[key], rel_tol=1e-6 if precision == "fp64" else 1e-2,
                                abs_tol=1e-12), (j, key)
