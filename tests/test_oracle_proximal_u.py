"""Pins of the oracle's U step with the proximal term h_i > 0 (eq.
proximalfunctionu): U^k minimizes mu_i/2 |J_i - U P_i + Lambda_i|^2 + h_i/2
|U - U^{k-1}|^2 over rotations.  Checked by brute force on the raw objective, by
the vanishing of its Riemannian gradient on SO(d), and in the limit h -> infinity,
where U stays at U^{k-1}.  The GPU path keeps h_i = 0 (every workload starts with
flipped elements, where Sec. 6 disables the term); these pins cover the oracle's
restatement of the paper's U step in full."""
import math

import numpy as np
import pytest
import scipy.optimize as so
from scipy.spatial.transform import Rotation

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def _mesh(d):
    rng = np.random.default_rng(21 + d)
    if d == 2:
        V, T = wk.grid_triangles(5, 4)
    else:
        V, T = wk.cube_tets(2)
    return V + rng.uniform(-0.03, 0.03, V.shape), T


def _state_before_u_step(d, h_scale):
    """Three iterations with the proximal weight h_i = h_scale w_i, then the
    inputs of the fourth U step: J, Lambda, P^{k-1}, U^{k-1}, mu, h."""
    V, T = _mesh(d)
    rng = np.random.default_rng(31 + d)
    W0 = V + 0.1 * rng.normal(size=V.shape)
    o0 = admm.Oracle(V, T, np.array([0, 1]), W0[:2], "sd", rho=2.0)
    o = admm.Oracle(V, T, np.array([0, 1]), W0[:2], "sd", rho=2.0, h=h_scale * o0.w)
    s = o.init(W0)
    for _ in range(3):
        s, _ = o.step(s)
    W = o.w_step(s)
    s1 = o.local_steps(s, W)
    return o, s, s1


def _objective(J, Lam, P0, U0, mu, h):
    return lambda U: 0.5 * mu * np.sum((J - U @ P0 + Lam) ** 2) + 0.5 * h * np.sum((U - U0) ** 2)


@pytest.mark.parametrize("d", [2, 3])
def test_u_step_minimizes_the_proximal_objective(d):
    o, s, s1 = _state_before_u_step(d, 4.0)
    for i in range(4):
        J, Lam, P0, U0, mu, h = s1.J[i], s.Lam[i], s.P[i], s.U[i], o.mu[i], o.h[i]
        assert h > 0
        F = _objective(J, Lam, P0, U0, mu, h)
        if d == 2:
            a = np.linspace(0, 2 * math.pi, 200001)
            Us = admm.rot2(np.cos(a), np.sin(a))
            vals = 0.5 * mu * np.sum((J[None] - Us @ P0 + Lam[None]) ** 2, axis=(1, 2)) + \
                0.5 * h * np.sum((Us - U0[None]) ** 2, axis=(1, 2))
            best = vals.min()
        else:
            Rs = Rotation.random(20000, random_state=17 + i).as_matrix()
            x0 = Rotation.from_matrix(Rs[int(np.argmin([F(R) for R in Rs]))]).as_rotvec()
            r = so.minimize(lambda v: F(Rotation.from_rotvec(v).as_matrix()), x0, method="Nelder-Mead",
                            options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
            best = r.fun
        U = s1.U[i]
        np.testing.assert_allclose(U.T @ U, np.eye(d), atol=1e-13)
        assert abs(np.linalg.det(U) - 1.0) < 1e-13
        assert F(U) <= best + 1e-9 * max(1.0, best)


@pytest.mark.parametrize("d", [2, 3])
def test_riemannian_gradient_of_the_proximal_objective_vanishes(d):
    """For F(U) = mu/2 |U P - A|^2 + h/2 |U - U0|^2 on SO(d), grad F = mu (U P - A) P
    + h (U - U0) and the minimizer has skew(U^T grad F) = 0."""
    o, s, s1 = _state_before_u_step(d, 4.0)
    for i in range(o.m):
        A = s1.J[i] + s.Lam[i]
        P0, U0, mu, h, U = s.P[i], s.U[i], o.mu[i], o.h[i], s1.U[i]
        G = mu * (U @ P0 - A) @ P0 + h * (U - U0)
        M = U.T @ G
        scale = mu * np.abs(A @ P0).max() + h
        assert np.abs(M - M.T).max() <= 1e-11 * scale


@pytest.mark.parametrize("d", [2, 3])
def test_large_proximal_weight_keeps_the_previous_rotation(d):
    """h_i -> infinity: the proximal term dominates and U^k = U^{k-1} up to O(mu/h)."""
    o, s, s1 = _state_before_u_step(d, 1e10)
    for i in range(o.m):
        assert np.abs(s1.U[i] - s.U[i]).max() < 1e-7
    # and h = 0 (no proximal term) moves U away from U^{k-1}
    o0, t, t1 = _state_before_u_step(d, 0.0)
    assert max(np.abs(t1.U[i] - t.U[i]).max() for i in range(o0.m)) > 1e-4


def test_h_bound_against_hand_values():
    """h_i = 4 w_i^2 B_i^2 / mu_i with B_i^2 = 5 (1 + |grad f(P_i)|^2) (Prop. 1 with gamma = 1,
    eps = 0; Sec. 6), worked by hand for w = 1/2, mu = 3/2:
      P = I (both energies): grad f = 0, B^2 = 5, h = 4 * 0.25 * 5 / 1.5 = 10/3;
      SD, P = diag(2, 1): grad f = P - P^-3 = diag(2 - 1/8, 0), |grad f|^2 = 3.515625,
          B^2 = 5 * 4.515625 = 22.578125, h = 22.578125 / 1.5;
      SG, P = diag(2, 1): grad f = P - P^-1 = diag(1.5, 0), B^2 = 5 * 3.25 = 16.25, h = 16.25 / 1.5."""
    from oracle import schedule
    w = np.array([0.5, 0.5])
    mu = np.array([1.5, 1.5])
    P = np.stack([np.eye(2), np.diag([2.0, 1.0])])
    hd = schedule.h_bound(P, w, mu, "sd")
    hg = schedule.h_bound(P, w, mu, "sg")
    assert math.isclose(hd[0], 10.0 / 3.0, rel_tol=1e-14) and math.isclose(hg[0], 10.0 / 3.0, rel_tol=1e-14)
    assert math.isclose(hd[1], 22.578125 / 1.5, rel_tol=1e-14)
    assert math.isclose(hg[1], 16.25 / 1.5, rel_tol=1e-14)
