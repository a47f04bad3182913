"""Pins of the oracle's symmetric ARAP energy, f_SA(X) = (|X - R|^2 + |X^-1 - R^-1|^2)/2
with R the rotation of X: one more rotation-invariant defining function plugged into
the same splitting (Sec. 3: other energies from the literature fit the framework;
the prox of a function of the singular values works eigenvalue by eigenvalue,
Supplemental "Solving the Optimization in P")."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def _phi(s):
    return 0.5 * ((s - 1.0) ** 2 + (1.0 / s - 1.0) ** 2)


@pytest.mark.parametrize("d", [2, 3])
def test_definition_equals_the_singular_value_form(d):
    """The definition (with R and the inverses) equals sum_k phi(s_k) for random
    unflipped matrices, and sI gives d phi(s)."""
    rng = np.random.default_rng(71 + d)
    A = rng.normal(size=(20, d, d))
    A[np.linalg.det(A) < 0, :, 0] *= -1
    s = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(admm.f_energy(A, "sa"), _phi(s).sum(axis=1), rtol=1e-12)
    for sc in (0.3, 1.0, 2.5):
        X = (sc * np.eye(d))[None]
        assert math.isclose(admm.f_energy(X, "sa")[0], d * _phi(sc), rel_tol=1e-13, abs_tol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_zero_exactly_at_rotations_and_rotation_invariant(d):
    rng = np.random.default_rng(81 + d)
    if d == 3:
        Rm = Rotation.random(6, random_state=5).as_matrix()
        Rn = Rotation.random(6, random_state=6).as_matrix()
    else:
        a, b = rng.uniform(0, 6, 6), rng.uniform(0, 6, 6)
        Rm, Rn = admm.rot2(np.cos(a), np.sin(a)), admm.rot2(np.cos(b), np.sin(b))
    assert np.abs(admm.f_energy(Rm, "sa")).max() < 1e-14
    assert np.abs(admm.grad_f(Rm, "sa")).max() < 1e-13
    A = rng.normal(size=(6, d, d))
    A[np.linalg.det(A) < 0, :, 0] *= -1
    np.testing.assert_allclose(admm.f_energy(Rm @ A @ Rn, "sa"), admm.f_energy(A, "sa"), rtol=1e-11)


def test_barrier_and_convexity_of_the_scalar_function():
    """phi grows without bound as s -> 0 (the flip barrier the scheme needs) and
    phi'' = 1 + (3 - 2s)/s^4 > 0 on s > 0 (unique scalar prox root)."""
    s = np.exp(np.linspace(-12, 6, 4001))
    assert _phi(s[0]) > 1e9
    d2 = 1.0 + (3.0 - 2.0 * s) / s ** 4
    assert d2.min() > 0.9
    # phi'' against second differences of phi
    h = 1e-4
    sm = np.array([0.2, 0.7, 1.0, 1.5, 2.0, 4.0])
    fd = (_phi(sm + h) - 2 * _phi(sm) + _phi(sm - h)) / h ** 2
    np.testing.assert_allclose(fd, 1.0 + (3.0 - 2.0 * sm) / sm ** 4, rtol=1e-5)


def test_scheme_unflips_and_meets_thresholds_with_the_symmetric_arap_energy():
    """From a disk map with flipped triangles the iteration with f_SA removes the
    flips, keeps every P_i SPD and the P-step stationarity w grad f(P) =
    mu symm(U^T Lambda) after each iteration, and meets the thresholds."""
    wl = wk.uv_disk(grid=20, seed=73, rho=3.0, energy="sa")
    assert wl.meta["flipped0"] > 0
    o = admm.Oracle.from_workload(wl)
    seen = []

    def cb(k, s0, s1, st):
        assert np.linalg.eigvalsh(s1.P).min() > 0
        lhs = o.w[:, None, None] * admm.grad_f(s1.P, "sa")
        rhs = o.mu[:, None, None] * admm.symm(np.transpose(s1.U, (0, 2, 1)) @ s1.Lam)
        assert np.abs(lhs - rhs).max() <= 1e-9 * max(1e-30, np.abs(lhs).max())
        seen.append(st)

    s, st = o.run(wl.W0, 600, callback=cb)
    assert st.converged and st.n_flipped == 0, (st.k, st.e_prim, st.thr_prim, st.n_flipped)
    assert seen[-1].e_prim < seen[0].e_prim * 1e-3
    assert math.isfinite(o.energy(s.W))
