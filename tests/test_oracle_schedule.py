"""Pins of the oracle's penalty schedule (Algorithm 2; Sec. 6, "Rescaling mu_i and
Lambda"; Lemma 1 and Proposition 1), each against what the paper and the
mathematics fix rather than against a retyped formula."""
import math

import numpy as np
import pytest

from oracle import admm, schedule
from paper_2107_05200_gb300 import workloads as wk


@pytest.mark.parametrize("B", [math.sqrt(5.0), 3.0, 10.0, 1e3, 1e6])
def test_lipschitz_constants_are_the_roots_of_lemma_1(B):
    b = np.array([B])
    cl = schedule.c_lipschitz(b, "sg")[0]
    clg = schedule.c_lipschitz(b, "sd")[0]
    # C^L: positive root of x^2 + B x - 1; C^LG: positive root of x^4 + B x^3 - 1
    assert abs(cl * cl + B * cl - 1.0) < 1e-14 * max(1.0, B)
    assert abs(clg ** 4 + B * clg ** 3 - 1.0) < 1e-13 * max(1.0, B)
    assert cl > 0 and clg > 0
    # Lemma 1: C^L <= C^LG <= 1
    assert cl <= clg <= 1.0


def test_mu_min_is_where_the_sufficient_decrease_coefficient_vanishes():
    # Proposition 1's proof needs (w + mu)/2 - 2 gamma w^2 F^2 / mu > 0 (gamma = 1,
    # eps = 0); mu_min is the boundary of that condition
    rng = np.random.default_rng(3)
    for energy in ("sd", "sg"):
        for d in (2, 3):
            A = rng.normal(size=(50, d, d))
            P = np.einsum("mij,mkj->mik", A, A) + 0.2 * np.eye(d)
            w = rng.uniform(0.01, 2.0, size=50)
            mu = schedule.mu_min(P, w, energy)
            B = np.sqrt(5.0 * (1.0 + schedule.grad_f_norm(P, energy) ** 2))
            F = schedule.lipschitz_F(B, energy, d)
            coef = lambda m: (w + m) / 2.0 - 2.0 * w * w * F * F / m
            assert np.all(np.abs(coef(mu)) < 1e-9 * w * F * F)
            assert np.all(coef(mu * 1.001) > 0) and np.all(coef(mu * 0.999) < 0)
            # mu_min >= w already (F >= 1): max(mu_min, w) = mu_min
            assert np.all(mu >= w)


def test_gradient_norm_from_eigenvalues():
    # for SPD P = E diag(p) E^T: grad f_SD has eigenvalues p - p^-3, grad f_SG p - 1/p
    rng = np.random.default_rng(4)
    for d in (2, 3):
        E = np.linalg.qr(rng.normal(size=(20, d, d)))[0]
        p = rng.uniform(0.3, 3.0, size=(20, d))
        P = np.einsum("mij,mj,mkj->mik", E, p, E)
        sd = np.sqrt(np.sum((p - p ** -3) ** 2, axis=1))
        sg = np.sqrt(np.sum((p - 1.0 / p) ** 2, axis=1))
        np.testing.assert_allclose(schedule.grad_f_norm(P, "sd"), sd, rtol=1e-10)
        np.testing.assert_allclose(schedule.grad_f_norm(P, "sg"), sg, rtol=1e-10)
        # at P = I (the rigid-motion fixed point) the gradient vanishes
        I = np.broadcast_to(np.eye(d), (3, d, d)).copy()
        assert np.all(schedule.grad_f_norm(I, "sd") < 1e-14)


def test_rescale_keeps_the_unscaled_multiplier_and_moves_mu_by_rho_over_2():
    mu = np.array([1.0, 1.0, 1.0, 1.0, 1.0])
    Lam = np.arange(5 * 4, dtype=float).reshape(5, 2, 2) + 1.0
    ep = np.array([10.0, 1.0, 1.0, 6.0, 1.0])
    ed = np.array([1.0, 10.0, 1.0, 1.0, 10.0])
    lo = np.array([0.1, 0.1, 0.1, 0.1, 0.7])
    new, L2 = schedule.rescale(mu, Lam, ep, ed, lo)
    np.testing.assert_allclose(new, [2.5, 0.4, 1.0, 2.5, 0.7])   # last: the lower bound binds
    np.testing.assert_allclose(new[:, None, None] * L2, mu[:, None, None] * Lam, rtol=1e-15)


def test_rescale_events():
    ev = schedule.rescale_iterations(600)
    # five directly after initialization, then gaps floor(5 * 1.5^p) with p = 5, 6, ...
    assert ev == [1, 2, 3, 4, 5, 42, 98, 183, 311, 503]


def test_paper_schedule_reaches_the_tolerance_flip_free_on_the_disk():
    """On the 48^2 disk, mu = w fixed stops at the 500-iteration cap; Algorithm 2
    with the rescaling reaches the termination test with no flipped triangle."""
    wl = wk.uv_disk()
    o = admm.Oracle.from_workload(wl)
    s, st, n_events = schedule.run(o, wl.W0, 500)
    assert st.converged and st.n_flipped == 0 and st.k < 500
    assert n_events >= 6
    # the KKT identity of the P step still holds with the rescaled penalties
    lhs = o.w[:, None, None] * admm.grad_f(s.P, wl.energy)
    rhs = o.mu[:, None, None] * admm.symm(np.transpose(s.U, (0, 2, 1)) @ s.Lam)
    assert np.abs(lhs - rhs).max() < 1e-8 * (1.0 + np.abs(lhs).max())


def test_elements_at_rest_are_not_rescaled_on_rounding_noise():
    # J = U P up to rounding and J = J_prev: both element errors count as zero, so
    # neither branch of the rule fires and mu keeps its value
    wl = wk.cube_deform(cells=2, seed=35)
    o = admm.Oracle.from_workload(wl)
    s0 = o.init(wl.V)                      # the rest pose: J = I
    s1 = o.local_steps(s0, wl.V.copy())
    ep, ed = schedule.element_errors(o, s0, s1)
    assert np.all(ep == 0.0) and np.all(ed == 0.0)
    new, L2 = schedule.rescale(o.mu, s1.Lam, ep, ed, 0.0 * o.mu)
    np.testing.assert_array_equal(new, o.mu)
