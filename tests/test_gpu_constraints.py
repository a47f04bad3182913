"""General linear constraints A W = b on the GPU (Sec. 4, W update: any feasible
A W = b) against the FP64 oracle's KKT solve: trajectories in both precisions,
constraint rows that touch pinned vertices and follow moved handles, exact
feasibility of every iterate, and the refusals of the C ABI."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _cube_centroid():
    """The cube with its bottom face pinned, the top face's centroid moved and two
    top vertices held at their rest offset: no top vertex is pinned."""
    wl = wk.cube_deform(cells=3, seed=46, angle_deg=0.0, shift_x=0.2)
    n = wl.V.shape[0]
    z = wl.V[:, 2]
    bottom = np.nonzero(z < 1e-9)[0]
    top = np.nonzero(z > 1 - 1e-9)[0]
    shift = np.array([0.2, 0.0, 0.1])
    rows = [np.zeros(n), np.zeros(n)]
    rows[0][top] = 1.0 / len(top)
    rows[1][top[0]], rows[1][top[-1]] = 1.0, -1.0
    A = sp.csr_matrix(np.array(rows))
    b = np.vstack([wl.V[top].mean(axis=0) + shift, wl.V[top[0]] - wl.V[top[-1]]])
    W0 = wl.V.copy()
    W0[top] += shift
    return wl, bottom, wl.V[bottom].copy(), A, b, W0


def _disk_rows():
    """A disk with its boundary pinned and three rows on interior vertices: a
    centroid of four, a link W_a - W_b = 0, and W_f - W_p = t tying an interior
    vertex to a pinned one (its pinned part moves to the right-hand side).  The
    start is the scaled square with the pins on the circle (36 flipped triangles,
    |det J| >= 1.4), so every element is far from the flip threshold; the start was
    chosen at a time when the disk generator could still leave one triangle
    degenerate to rounding, which it no longer does."""
    wl = wk.uv_disk(grid=12, seed=61, rho=3.0)
    n = wl.V.shape[0]
    W0 = 1.4 * (wl.V - 0.5)
    W0[wl.pins] = wl.pin_pos
    pinned = set(int(p) for p in wl.pins)
    interior = [v for v in range(n) if v not in pinned]
    rows, b = [], []
    r = np.zeros(n)
    r[interior[10:14]] = 0.25
    rows.append(r)
    b.append(W0[interior[10:14]].mean(axis=0) + np.array([0.02, -0.01]))
    r = np.zeros(n)
    r[interior[30]], r[interior[45]] = 1.0, -1.0
    rows.append(r)
    b.append(np.zeros(2))
    p = int(wl.pins[5])
    f = interior[0]
    r = np.zeros(n)
    r[f], r[p] = 1.0, -1.0
    rows.append(r)
    b.append(wl.V[f, :2] - wl.V[p, :2])
    return wl, sp.csr_matrix(np.array(rows)), np.array(b), W0


def _oracle(V, T, pins, pin_pos, energy, rho, A, b, W0, iters):
    o = admm.Oracle(V, T, pins, pin_pos, energy, rho, constraints=(A, b))
    s = o.init(W0)
    hist = []
    for _ in range(iters):
        s, st = o.step(s)
        hist.append(st)
    return s, hist


def test_cube_centroid_fp64_trajectory_matches_the_oracle():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl, pins, pin_pos, A, b, W0 = _cube_centroid()
    iters = 25
    s, hist = _oracle(wl.V, wl.T, pins, pin_pos, wl.energy, 3.0, A, b, W0, iters)
    with Solver(wl.V, wl.T, pins, pin_pos, energy=wl.energy, rho=3.0, precision="fp64", check_every=5) as sol:
        sol.set_constraints(A, b)
        sol.init(W0)
        st = sol.iterate(iters, stop_at_tol=False)
        W = sol.W()
        U, P, L = sol.state()
    np.testing.assert_allclose(A @ W, b, rtol=0, atol=1e-11)
    np.testing.assert_allclose(W[pins], pin_pos, rtol=0, atol=0)
    assert _rel(W, s.W) < 1e-8
    assert _rel(P, s.P) < 1e-7
    assert _rel(L, s.Lam) < 1e-6
    ref = hist[-1]
    assert math.isclose(st["e_prim"], ref.e_prim, rel_tol=1e-6, abs_tol=1e-12)
    assert math.isclose(st["energy_P"], ref.energy_P, rel_tol=1e-9)
    assert st["n_flipped"] == ref.n_flipped


@pytest.mark.parametrize("precision,wtol", [("fp64", 1e-8), ("fp32", 1e-5)])
def test_disk_rows_on_pinned_vertices_follow_moved_handles(precision, wtol):
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl, A, b, W0 = _disk_rows()
    iters = 20
    moved = wl.pin_pos + 0.03 * np.stack([np.cos(np.arange(len(wl.pins))), np.sin(np.arange(len(wl.pins)))], 1)
    with Solver.from_workload(wl, precision=precision, check_every=5) as sol:
        sol.set_constraints(A, b)
        sol.init(W0)
        sol.iterate(iters, stop_at_tol=False)
        W1 = sol.W()
        sol.set_handles(moved)
        sol.iterate(iters, stop_at_tol=False)
        W2 = sol.W()
    o = admm.Oracle.from_workload(wl, constraints=(A, b))
    s1, _ = o.run(W0, iters, stop_at_tol=False)
    np.testing.assert_allclose(A @ W1, b, rtol=0, atol=1e-11)
    assert _rel(W1, s1.W) < wtol
    # the continuation after the handles moved: the oracle with the moved pins,
    # started from the first leg's state
    o2 = admm.Oracle(wl.V, wl.T, wl.pins, moved, wl.energy, wl.rho, constraints=(A, b))
    s2 = s1
    for _ in range(iters):
        s2, _ = o2.step(s2)
    np.testing.assert_allclose(A @ W2, b, rtol=0, atol=1e-11)
    np.testing.assert_allclose(W2[wl.pins], moved, rtol=0, atol=0)
    assert _rel(W2, s2.W) < wtol


def test_fp32_cube_centroid_converges_flip_free_and_feasible():
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl, pins, pin_pos, A, b, W0 = _cube_centroid()
    o = admm.Oracle(wl.V, wl.T, pins, pin_pos, wl.energy, 3.0, constraints=(A, b))
    so, sto = o.run(W0, 400)
    with Solver(wl.V, wl.T, pins, pin_pos, energy=wl.energy, rho=3.0, precision="fp32", check_every=10) as sol:
        sol.set_constraints(A, b)
        sol.init(W0)
        st = sol.iterate(400)
        W = sol.W()
    assert st["converged"] == 1 and st["n_flipped"] == 0
    np.testing.assert_allclose(A @ W, b, rtol=0, atol=1e-11)
    assert abs(st["checked_iter"] - sto.k) <= 10
    assert math.isclose(o.energy(W), o.energy(so.W), rel_tol=1e-4)


def test_refusals():
    _need_gpu()
    from paper_2107_05200_gb300._native import FFAError
    from paper_2107_05200_gb300.solver import Solver
    wl, A, b, W0 = _disk_rows()
    n = wl.V.shape[0]
    with Solver.from_workload(wl, precision="fp64") as sol:
        # a row on pinned vertices only, and a row repeated: dependent
        r = np.zeros((1, n))
        r[0, wl.pins[0]] = 1.0
        with pytest.raises(FFAError, match="depends"):
            sol.set_constraints(sp.csr_matrix(r), np.zeros((1, 2)))
        with pytest.raises(FFAError, match="depends"):
            sol.set_constraints(sp.vstack([A, A[1]]), np.vstack([b, b[1:2]]))
        with pytest.raises(FFAError, match="c <= 256"):
            sol.set_constraints(sp.csr_matrix((257, n)), np.zeros((257, 2)))
        sol.set_constraints(A, b)
        with pytest.raises(FFAError, match="already"):
            sol.set_constraints(A, b)
        sol.init(W0)
        with pytest.raises(FFAError, match="pinned constraints only"):
            sol.forward_unrolled(3, 1)
        with pytest.raises(FFAError, match="multiplier"):
            sol.wstep_residual()
    with Solver.from_workload(wl, precision="fp64") as sol:
        sol.init(W0)
        with pytest.raises(FFAError, match="before ffa_init"):
            sol.set_constraints(A, b)
    with Solver(wl.V, wl.T, None, None, energy="sd", rho=3.0) as sol:
        with pytest.raises(FFAError, match="pinned vertex"):
            sol.set_constraints(A, b)
    with Solver.from_workload(wl, penalties="paper") as sol:
        with pytest.raises(FFAError, match="penalty schedule"):
            sol.set_constraints(A, b)
