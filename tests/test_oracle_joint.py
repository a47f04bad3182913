"""Pins of the oracle's joint (U, P) prox variant (not the paper's scheme; the
paper's Algorithm 1 updates U with P^{k-1}, then P)."""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def _objective(U, P, A, w, mu, energy):
    R = U @ P - A
    return w * admm.f_energy(P, energy) + 0.5 * mu * np.einsum("mij,mij->m", R, R)


def _random_rotation(rng, d, k):
    Q, Rr = np.linalg.qr(rng.normal(size=(k, d, d)))
    Q = Q * np.sign(np.einsum("mii->mi", Rr))[:, None, :]
    Q[np.linalg.det(Q) < 0, :, 0] *= -1
    return Q


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("energy", ["sd", "sg"])
def test_joint_step_is_the_joint_minimizer(d, energy):
    rng = np.random.default_rng(21 + d)
    k = 40
    A = rng.normal(size=(k, d, d))
    A[: k // 4] *= -1.0                      # some with det A < 0
    w = rng.uniform(0.1, 2.0, k)
    mu = rng.uniform(0.5, 5.0, k)
    U = admm.procrustes(A, np.broadcast_to(np.eye(d), (k, d, d)).copy())
    P = admm.p_step(admm.symm(np.transpose(U, (0, 2, 1)) @ A), w, mu, energy)
    best = _objective(U, P, A, w, mu, energy)
    # alternating minimization from random starts never does better
    for _ in range(3):
        Ua = _random_rotation(rng, d, k)
        for _ in range(200):
            Pa = admm.p_step(admm.symm(np.transpose(Ua, (0, 2, 1)) @ A), w, mu, energy)
            Ua = admm.procrustes(A @ Pa, Ua)
        Pa = admm.p_step(admm.symm(np.transpose(Ua, (0, 2, 1)) @ A), w, mu, energy)
        assert np.all(best <= _objective(Ua, Pa, A, w, mu, energy) + 1e-9 * (1 + np.abs(best)))
    # nor do small perturbations of (U, P)
    for _ in range(20):
        dR = _random_rotation(rng, d, k)
        dR = np.array([np.linalg.matrix_power(r, 1) for r in dR])
        small = admm.procrustes(np.eye(d) + 1e-3 * (dR - np.eye(d)), np.broadcast_to(np.eye(d), (k, d, d)).copy())
        E = rng.normal(size=(k, d, d)) * 1e-4
        Pp = P + admm.symm(E)
        assert np.all(best <= _objective(U @ small, Pp, A, w, mu, energy) + 1e-12 * (1 + np.abs(best)))


def test_joint_variant_keeps_rigid_motions_fixed_and_converges():
    wl = wk.uv_disk(grid=16, seed=22)
    o = admm.Oracle.from_workload(wl, local_variant="joint")
    s, st = o.run(wl.W0, 500)
    assert st.converged and st.n_flipped == 0
    # a rotation of the source is a fixed point: J in SO(2), Lambda = 0 -> U = J, P = I
    th = 0.3
    Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    W = wl.V @ Rm.T
    s0 = o.init(W)
    s1 = o.local_steps(s0, W)
    assert np.abs(s1.P - np.eye(2)).max() < 1e-12 and np.abs(s1.Lam).max() < 1e-12
