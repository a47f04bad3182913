"""Pins of the oracle's Tutte initializer (App. A, "Tutte's Energy")."""
import numpy as np
import pytest

from oracle import tutte as ot
from paper_2107_05200_gb300 import workloads as wk


def _disk(grid, seed):
    wl = wk.uv_disk(grid=grid, seed=seed, target_flip=None, sigma=0.0)
    return wl.V, wl.T, wl.pins, wl.pin_pos


def test_minimizer_matches_a_generic_optimizer_on_the_energy_as_defined():
    scipy_opt = pytest.importorskip("scipy.optimize")
    V, T, b, bp = _disk(5, 11)
    W = ot.tutte(V, T, b, bp)
    inner = np.setdiff1d(np.arange(V.shape[0]), b)

    def energy(x):
        Wx = W.copy()
        Wx[inner] = x.reshape(-1, 2)
        return ot.tutte_energy(V, T, Wx)

    rng = np.random.default_rng(12)
    x0 = rng.normal(size=(len(inner), 2)).ravel()
    res = scipy_opt.minimize(energy, x0, method="L-BFGS-B", options={"maxiter": 20000, "gtol": 1e-12, "ftol": 1e-15})
    np.testing.assert_allclose(res.x.reshape(-1, 2), W[inner], atol=1e-5)
    assert energy(W[inner].ravel()) <= res.fun + 1e-12


def test_interior_vertices_are_weighted_averages_of_their_neighbours():
    V, T, b, bp = _disk(7, 13)
    W = ot.tutte(V, T, b, bp)
    nbr = {}
    for tri in np.asarray(T):
        for a in range(3):
            for c in range(3):
                if a != c:
                    nbr.setdefault(int(tri[a]), set()).add(int(tri[c]))
    fixed = set(int(v) for v in b)
    for i, js in nbr.items():
        if i in fixed:
            continue
        num = np.zeros(2)
        den = 0.0
        for j in js:
            c = 1.0 / np.linalg.norm(V[i] - V[j])
            num += c * W[j]
            den += c
        np.testing.assert_allclose(W[i], num / den, atol=1e-12)
    np.testing.assert_array_equal(W[b], bp)


def test_tuttes_theorem_convex_boundary_gives_no_flipped_triangle():
    V, T, b, bp = _disk(24, 14)
    W = ot.tutte(V, T, b, bp)
    assert wk.flipped_fraction(W, T) == 0.0
