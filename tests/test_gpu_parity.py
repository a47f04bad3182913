"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the FP64 local step must follow the oracle's trajectory to ~1e-8
relative (its only difference is the float factor inside the refined W step);
the FP32 local step must keep vertex positions within 1e-5 relative and the
energy within 1e-6 relative of the oracle (the precision split of the local
step in float and the global/reduction work in double).
"""
import math

import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _solver(wl, **kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05200_gb300.solver import Solver
    return Solver.from_workload(wl, **kw)


def _oracle_run(wl, iters):
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    hist = []
    for _ in range(iters):
        s1, st = o.step(s)
        hist.append(st)
        s = s1
    return o, s, hist


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _small_workloads():
    return {
        "disk2d_sd": wk.uv_disk(grid=14, seed=31),
        "surface_sg": wk.uv_heightfield(grid=18, seed=32),
        "cube3d_sd": wk.cube_deform(cells=4, seed=33),
        "cube3d_sg": wk.cube_deform(cells=3, seed=34, energy="sg"),
    }


@pytest.mark.parametrize("name", ["disk2d_sd", "surface_sg", "cube3d_sd", "cube3d_sg"])
def test_polar_init_matches(name):
    wl = _small_workloads()[name]
    o = admm.Oracle.from_workload(wl)
    s0 = o.init(wl.W0)
    with _solver(wl, precision="fp64") as sol:
        sol.init(wl.W0)
        U, P, L = sol.state()
        W = sol.W()
    np.testing.assert_allclose(W, s0.W, rtol=0, atol=1e-15)
    assert _rel(P, s0.P) < 1e-10
    assert _rel(U, s0.U) < 1e-10
    assert np.abs(L).max() == 0.0


@pytest.mark.parametrize("name", ["disk2d_sd", "surface_sg", "cube3d_sd", "cube3d_sg"])
def test_fp64_trajectory_matches(name):
    wl = _small_workloads()[name]
    iters = 25
    o, s, hist = _oracle_run(wl, iters)
    with _solver(wl, precision="fp64", check_every=5) as sol:
        sol.init(wl.W0)
        st = sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    assert _rel(W, s.W) < 1e-8
    assert _rel(P, s.P) < 1e-7
    assert _rel(L, s.Lam) < 1e-6
    ref = hist[-1]
    assert math.isclose(st["e_prim"], ref.e_prim, rel_tol=1e-6, abs_tol=1e-12)
    assert math.isclose(st["e_dual"], ref.e_dual, rel_tol=1e-5, abs_tol=1e-12)
    assert math.isclose(st["thr_dual"], ref.thr_dual, rel_tol=1e-8)
    assert math.isclose(st["thr_prim"], ref.thr_prim, rel_tol=1e-8)
    assert math.isclose(st["energy_P"], ref.energy_P, rel_tol=1e-9)
    assert st["n_flipped"] == ref.n_flipped


@pytest.mark.parametrize("name", ["disk2d_sd", "surface_sg", "cube3d_sd"])
def test_fp32_trajectory_within_stated_tolerance(name):
    wl = _small_workloads()[name]
    iters = 25
    o, s, hist = _oracle_run(wl, iters)
    with _solver(wl, precision="fp32", check_every=5) as sol:
        sol.init(wl.W0)
        st = sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
        E = sol.energy()
    assert _rel(W, s.W) < 1e-5
    Eo = o.energy(s.W)
    if math.isfinite(Eo):
        assert math.isclose(E, Eo, rel_tol=1e-6)
    assert math.isclose(st["energy_P"], hist[-1].energy_P, rel_tol=1e-5)


def test_uv_disk_full_size_fp64_and_fp32():
    """The 48x48 uv-disk workload, 500 iterations (its iteration cap), both precisions."""
    wl = wk.uv_disk()
    o, s, hist = _oracle_run(wl, 500)
    for prec, tol in (("fp64", 1e-8), ("fp32", 1e-5)):
        with _solver(wl, precision=prec, check_every=50) as sol:
            sol.init(wl.W0)
            st = sol.iterate(500, stop_at_tol=False)
            W = sol.W()
        assert _rel(W, s.W) < tol, prec
        assert st["n_flipped"] == hist[-1].n_flipped == 0


def test_converges_to_tolerance_and_stops():
    """rho = 3 uv-disk: the GPU loop stops at the same check as the oracle, flip-free."""
    wl = wk.uv_disk(grid=24, seed=22, rho=3.0)
    o = admm.Oracle.from_workload(wl)
    s, st_o = o.run(wl.W0, 400)
    with _solver(wl, precision="fp64", check_every=1) as sol:
        sol.init(wl.W0)
        st = sol.iterate(400, stop_at_tol=True)
        W = sol.W()
    assert st["converged"] == 1 and st_o.converged
    assert st["iters"] == st_o.k
    assert _rel(W, s.W) < 1e-8


@pytest.mark.parametrize("energy", ["sd", "sg"])
def test_energy_and_gradient(energy):
    wl = wk.cube_deform(cells=3, seed=35, energy=energy)
    rng = np.random.default_rng(3)
    W = wl.V + 0.01 * rng.normal(size=wl.V.shape)
    o = admm.Oracle.from_workload(wl)
    for prec, etol, gtol in (("fp64", 1e-12, 1e-10), ("fp32", 1e-6, 1e-4)):
        with _solver(wl, precision=prec) as sol:
            E = sol.energy(W)
            G = sol.gradient(W)
            assert math.isclose(E, o.energy(W), rel_tol=etol)
            assert _rel(G, o.energy_gradient(W)) < gtol
            Wf = W.copy()
            Wf[:, 0] *= -1
            assert sol.energy(Wf) == math.inf


def test_wstep_residual_is_small():
    wl = wk.cube_deform(cells=6, seed=36)
    with _solver(wl, precision="fp32") as sol:
        sol.init(wl.W0)
        sol.iterate(3, stop_at_tol=False)
        r = sol.wstep_residual()
    assert r < 1e-9


def test_no_pins_fixes_vertex_zero_and_single_element():
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
    T = np.array([[0, 1, 2]], np.int32)
    W0 = V * 1.3 + 0.1
    o = admm.Oracle(V, T, np.array([], int), np.zeros((0, 2)), "sd")
    s = o.init(W0)
    for _ in range(5):
        s, _ = o.step(s)
    with _solver(wk.Workload("tri", V, T, np.zeros(0, np.int32), np.zeros((0, 2)), W0, "sd"),
                 precision="fp64") as sol:
        sol.init(W0)
        sol.iterate(5, stop_at_tol=False)
        W = sol.W()
    np.testing.assert_array_equal(W[0], [0.0, 0.0])
    assert _rel(W, s.W) < 1e-9


def test_invalid_inputs_are_rejected():
    from paper_2107_05200_gb300._native import FFAError
    wl = wk.uv_disk(grid=6)
    bad = wk.Workload("bad", wl.V, wl.T.copy(), wl.pins, wl.pin_pos, wl.W0, "sd")
    bad.T[0, 1] = bad.T[0, 0]   # zero-area element
    with pytest.raises(FFAError, match="DEGENERATE"):
        _solver(bad)
    bad2 = wk.Workload("bad2", wl.V, wl.T, np.r_[wl.pins, wl.pins[:1]].astype(np.int32),
                       np.r_[wl.pin_pos, wl.pin_pos[:1]], wl.W0, "sd")
    with pytest.raises(FFAError, match="INVALID_ARG"):
        _solver(bad2)
    bad3 = wk.Workload("bad3", wl.V, wl.T.copy(), wl.pins, wl.pin_pos, wl.W0, "sd")
    bad3.T[3, 2] = wl.n + 5
    with pytest.raises(FFAError, match="INVALID_ARG"):
        _solver(bad3)
    with _solver(wl) as sol:
        with pytest.raises(FFAError, match="NOT_INITIALIZED"):
            sol.iterate(1)
        W0 = wl.W0.copy()
        W0[20] = np.nan
        sol.init(W0)
        with pytest.raises(FFAError, match="NAN"):
            sol.iterate(2, stop_at_tol=False)


@pytest.mark.parametrize("seed", [7, 61, 62, 63, 64, 65])
def test_disk_trajectory_for_any_seed(seed):
    """The generated starts hold no element at det J = 0 to rounding, so the GPU and the oracle
    take the same branch of eq. polardecompositionapplied for every element, whatever the seed."""
    wl = wk.uv_disk(grid=12, seed=seed)
    iters = 25
    o, s, hist = _oracle_run(wl, iters)
    with _solver(wl, precision="fp64", check_every=5) as sol:
        sol.init(wl.W0)
        sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    assert _rel(W, s.W) < 1e-8
    assert _rel(P, s.P) < 1e-7
    assert _rel(L, s.Lam) < 1e-6


def test_cube_deform_recipe_fp64_trajectory_200_iterations():
    """The benchmark's recipe (jittered cube, bottom fixed, top rotated 45 degrees and shifted,
    symmetric Dirichlet, mu = 3 w) at 16^3 cells (24,576 tets): 200 iterations of the FP64 GPU
    path against the oracle, W within 1e-8."""
    wl = wk.cube_deform(cells=16)
    iters = 200
    o, s, hist = _oracle_run(wl, iters)
    with _solver(wl, precision="fp64", check_every=50) as sol:
        sol.init(wl.W0)
        st = sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    err = _rel(W, s.W)
    print(f"\ncube 16^3, {iters} iterations: W rel. err {err:.3e}, P {_rel(P, s.P):.3e}, "
          f"Lambda {_rel(L, s.Lam):.3e}; e_prim {st['e_prim']:.3e} (oracle {hist[-1].e_prim:.3e}), "
          f"flips {st['n_flipped']} (oracle {hist[-1].n_flipped})")
    assert err < 1e-8
    assert st["n_flipped"] == hist[-1].n_flipped
    assert math.isclose(st["e_prim"], hist[-1].e_prim, rel_tol=1e-5)
