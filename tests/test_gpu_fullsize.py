"""Parity at the full workload sizes, in the launch configuration the benchmark
times (FP32 local step, two refinement sweeps).

The oracle cannot run these meshes end to end, so each check uses what it can
compute one element at a time or what holds at any size:
* the local step of one GPU iteration, recomputed by the oracle for sampled
  elements from the GPU's own inputs (W^{k+1} and the state after iteration k);
* the W step's residual |L_FF W_F - b_F| / |b_F| in double;
* flip-freeness of every P_i (all eigenvalues positive).
"""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sampled_local_step(wl, iters, n_sample, seed):
    from paper_2107_05200_gb300.solver import Solver
    with Solver.from_workload(wl, precision="fp32", refine_sweeps=2, check_every=50) as sol:
        sol.init(wl.W0)
        sol.iterate(iters, stop_at_tol=False)
        U0, P0, L0 = sol.state()
        sol.iterate(1, stop_at_tol=False)
        W1 = sol.W()
        U1, P1, L1 = sol.state()
        resid = sol.wstep_residual()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(wl.m, size=n_sample, replace=False))
    T = wl.T[idx].astype(np.int64)
    g, w = admm.element_gradients(wl.V, T)
    mu = wl.rho * w
    J = admm.jacobians(g, T, W1)
    A = J + L0[idx]
    U = admm.procrustes(A @ P0[idx], U0[idx])
    S = admm.symm(np.transpose(U, (0, 2, 1)) @ A)
    P = admm.p_step(S, w, mu, wl.energy)
    Lam = L0[idx] + J - U @ P
    return resid, (U1[idx], P1[idx], L1[idx], P1), (U, P, Lam), J


def _check(wl, iters):
    resid, gpu, ref, J = _sampled_local_step(wl, iters, 4000, 61)
    Ug, Pg, Lg, Pall = gpu
    Ur, Pr, Lr = ref
    assert resid < 1e-9
    # flip-free local output everywhere (eigenvalues of every P_i positive)
    assert np.linalg.eigvalsh(Pall).min() > 0
    scale = np.abs(J).max(axis=(1, 2)) + np.abs(Lr).max(axis=(1, 2)) + 1.0
    errP = np.abs(Pg - Pr).max(axis=(1, 2)) / scale
    errL = np.abs(Lg - Lr).max(axis=(1, 2)) / scale
    errU = np.abs(Ug - Ur).max(axis=(1, 2))
    # float inputs (W, U, P, Lambda rounded to float) and float arithmetic: a few
    # ulps of the element's scale, more where the rotation is ill-conditioned
    assert np.quantile(errP, 0.99) < 1e-5 and np.quantile(errL, 0.99) < 1e-5
    assert np.quantile(errU, 0.99) < 1e-4
    assert errP.max() < 1e-2 and errL.max() < 1e-2


def test_cube_deform_64_sampled_local_step_and_residual():
    """1,572,864 tets, the benchmark workload and launch configuration."""
    _need_gpu()
    _check(wk.cube_deform(), iters=20)


def test_uv_heightfield_512_sampled_local_step_and_residual():
    """522,242 intrinsic triangles, symmetric gradient energy."""
    _need_gpu()
    _check(wk.uv_heightfield(), iters=20)
