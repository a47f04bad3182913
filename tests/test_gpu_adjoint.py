"""Differentiation through unrolled iterations: the CUDA adjoint against central
finite differences of the FP64 oracle (small meshes, every pin coordinate) and of
the GPU's own double-precision forward (the 32^3-cell handle workload).

The loss is the mean squared distance of seeded interior vertices of W^K to the
bend-map targets; dL/db is taken for all pinned positions b.
"""
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
    return torch


def _loss_and_grad(W, wl):
    idx = wl.meta["target_idx"]
    diff = W[idx] - wl.meta["targets"]
    L = float(np.mean(np.sum(diff * diff, axis=1)))
    G = np.zeros_like(W)
    G[idx] = 2.0 * diff / len(idx)
    return L, G


def _oracle_loss(o, wl, b, K):
    o.wstep.pin_pos = np.asarray(b, np.float64)
    s = o.init(wl.W0)
    for _ in range(K):
        s, _ = o.step(s)
    return _loss_and_grad(s.W, wl)[0]


def _gpu_grad(wl, precision, K, ckpt):
    from paper_2107_05200_gb300.solver import Solver
    with Solver.from_workload(wl, precision=precision) as sol:
        sol.set_handles(wl.pin_pos)
        sol.init(wl.W0)
        sol.forward_unrolled(K, ckpt)
        W = sol.W()
        L, G = _loss_and_grad(W, wl)
        gb = sol.backward_unrolled(G)
        W_again = sol.W()
    return L, gb, W, W_again


def _small():
    # handles half-way along the bend: the 12-iteration map is far from the rest pose
    return wk.cube_handles(cells=4, seed=51, n_targets=12, lattice_start=1, lattice_step=2, pre_bend=0.5)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_adjoint_matches_oracle_central_differences(precision, tol):
    _need_gpu()
    wl = _small()
    K, ckpt = 12, 5            # segments of 5, 5 and 2 iterations
    L, gb, W, W_again = _gpu_grad(wl, precision, K, ckpt)
    np.testing.assert_array_equal(W, W_again)     # backward restores the final state
    o = admm.Oracle.from_workload(wl)
    L_o = _oracle_loss(o, wl, wl.pin_pos, K)
    assert math.isclose(L, L_o, rel_tol=1e-5 if precision == "fp32" else 1e-9)
    h = 1e-4
    fd = np.zeros_like(wl.pin_pos)
    for p in range(wl.pin_pos.shape[0]):
        for c in range(3):
            bp = wl.pin_pos.copy()
            bp[p, c] += h
            bm = wl.pin_pos.copy()
            bm[p, c] -= h
            fd[p, c] = (_oracle_loss(o, wl, bp, K) - _oracle_loss(o, wl, bm, K)) / (2 * h)
    err = np.linalg.norm(gb - fd) / np.linalg.norm(fd)
    assert err < tol, err


def test_adjoint_single_segment_equals_checkpointed():
    _need_gpu()
    wl = _small()
    _, g1, _, _ = _gpu_grad(wl, "fp64", 10, 10)
    _, g2, _, _ = _gpu_grad(wl, "fp64", 10, 3)
    np.testing.assert_allclose(g2, g1, rtol=1e-9, atol=1e-13)


def test_autograd_function_matches_direct_backward():
    torch = _need_gpu()
    from paper_2107_05200_gb300.autograd import unrolled_solve
    from paper_2107_05200_gb300.solver import Solver
    wl = _small()
    K = 8
    with Solver.from_workload(wl, precision="fp64") as sol:
        b = torch.tensor(wl.pin_pos, dtype=torch.float64, device="cuda", requires_grad=True)
        W0 = torch.tensor(wl.W0, dtype=torch.float64, device="cuda")
        idx = torch.tensor(wl.meta["target_idx"], dtype=torch.long, device="cuda")
        tgt = torch.tensor(wl.meta["targets"], dtype=torch.float64, device="cuda")
        W = unrolled_solve(b, sol, W0, K, 3)
        loss = ((W[idx] - tgt) ** 2).sum(dim=1).mean()
        loss.backward()
        g_auto = b.grad.cpu().numpy()
    _, g_direct, _, _ = _gpu_grad(wl, "fp64", K, 3)
    np.testing.assert_allclose(g_auto, g_direct, rtol=1e-9, atol=1e-13)


def test_handle_workload_full_size_directional_derivatives():
    """32^3 cells, 64 handles at rest, 200 iterations, checkpoints every 20.  The
    FP64 and FP32 adjoints' directional derivatives against central differences
    (h = 1e-4) of the FP64 forward along random handle directions, within
    1e-5 |g| |v| and 1e-4 |g| |v| (a projection can be much smaller than |g| |v|,
    and the difference quotient's own truncation error is of order 1e-7 absolute
    here); the FP32 handle gradient within 1e-4 of the FP64 one in relative norm.  (With the handles pre-bent, 200
    iterations do not reach the contractive regime and central differences at
    h = 1e-3, 1e-4, 1e-5 disagree in sign: that map has no gradient to check.)"""
    _need_gpu()
    from paper_2107_05200_gb300.solver import Solver
    wl = wk.cube_handles()
    K, ckpt = 200, 20
    _, gb, _, _ = _gpu_grad(wl, "fp32", K, ckpt)
    _, gb64, _, _ = _gpu_grad(wl, "fp64", K, ckpt)
    nb = wl.meta["n_bottom"]
    gh32, gh64 = gb[nb:], gb64[nb:]
    assert np.linalg.norm(gh32 - gh64) <= 1e-4 * np.linalg.norm(gh64)
    rng = np.random.default_rng(52)
    h = 1e-4
    with Solver.from_workload(wl, precision="fp64") as sol:
        def loss(b):
            sol.set_handles(b)
            sol.init(wl.W0)
            sol.iterate(K, stop_at_tol=False)
            return _loss_and_grad(sol.W(), wl)[0]
        for _ in range(2):
            v = np.zeros_like(wl.pin_pos)
            v[nb:] = rng.normal(size=(len(wl.pin_pos) - nb, 3))
            fd = (loss(wl.pin_pos + h * v) - loss(wl.pin_pos - h * v)) / (2 * h)
            ad = float(np.sum(gb * v))
            ad64 = float(np.sum(gb64 * v))
            assert abs(ad64 - fd) <= 1e-5 * np.linalg.norm(gh64) * np.linalg.norm(v), (ad64, fd)
            assert abs(ad - fd) <= 1e-4 * np.linalg.norm(gh64) * np.linalg.norm(v), (ad, fd)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_bent_handles_directional_derivatives_against_the_oracle(precision, tol):
    """Handles a quarter of the way along the bend on an 8^3-cell cube (16 handles,
    40 targets): 100 iterations reach the fixed point (the oracle's e_prim falls to
    1e-13), so the loss is a smooth function of the handle positions.  The adjoint's
    directional derivatives along random handle directions against central
    differences (h = 1e-4) of the FP64 oracle, within tol |g_handles| |v|."""
    _need_gpu()
    wl = wk.cube_handles(cells=8, seed=53, n_targets=40, lattice_start=1, lattice_step=2, pre_bend=0.25)
    K, ckpt = 100, 20
    _, gb, _, _ = _gpu_grad(wl, precision, K, ckpt)
    nb = wl.meta["n_bottom"]
    o = admm.Oracle.from_workload(wl)
    rng = np.random.default_rng(54)
    h = 1e-4
    for _ in range(2):
        v = np.zeros_like(wl.pin_pos)
        v[nb:] = rng.normal(size=(len(wl.pin_pos) - nb, 3))
        fd = (_oracle_loss(o, wl, wl.pin_pos + h * v, K) - _oracle_loss(o, wl, wl.pin_pos - h * v, K)) / (2 * h)
        ad = float(np.sum(gb * v))
        assert abs(ad - fd) <= tol * np.linalg.norm(gb[nb:]) * np.linalg.norm(v), (ad, fd)
