"""The oracle's iterates against Proposition 1 of the paper (Sec. 5, sufficient
decrease): with penalties mu_i above the bound built from Lemma 1's local
Lipschitz constant F_i, the proximal weight h_i >= 4 gamma w_i^2 B_i^2 / mu_i + 2 eps
and 0 < eps < min_i w_i / 2, every step k -> k+1 at which Conditions 1
(|grad f(P_i)| <= B_i at both iterates) and 2 (the Lambda step bounded by gamma)
hold satisfies

    Phi^{k+1} - Phi^k <= -lambda_min(L)/2 |W^{k+1} - W^k|^2
                         - eps sum_i (|U_i^{k+1} - U_i^k|^2 + |P_i^{k+1} - P_i^k|^2),

Phi the augmented Lagrangian of eq. augmentedlagrangian and L the W step's
operator on the free vertices.  Phi, the conditions and the bound are written
out here from their definitions; the oracle supplies only the iterates (and
Lemma 1's F_i, pinned separately).  A sign error in the W step's right-hand side,
or a P step that drops Lambda, breaks the bound at almost every step.  No GPU is
used."""
import numpy as np
import pytest

from oracle import admm, schedule
from paper_2107_05200_gb300 import workloads as wk


def _phi(o, s):
    """eq. augmentedlagrangian: sum_i w_i f(P_i) + mu_i/2 (|(GW)_i - U_i P_i + Lambda_i|^2 - |Lambda_i|^2)."""
    R = s.J - s.U @ s.P + s.Lam
    sq = lambda X: np.einsum("mij,mij->m", X, X)
    return float(np.sum(o.w * admm.f_energy(s.P, o.energy_name)) + 0.5 * np.sum(o.mu * (sq(R) - sq(s.Lam))))


def _gnorm(P, energy):
    G = admm.grad_f(P, energy)
    return np.sqrt(np.einsum("mij,mij->m", G, G))


CASES = {
    "disk_sd": lambda: wk.uv_disk(grid=8, seed=3, target_flip=None, sigma=0.003),
    "disk_sg": lambda: wk.uv_disk(grid=8, seed=3, target_flip=None, sigma=0.003, energy="sg"),
    "cube_sd": lambda: wk.cube_deform(cells=3, seed=5, angle_deg=10.0, shift_x=0.05),
    "cube_sg": lambda: wk.cube_deform(cells=3, seed=5, angle_deg=10.0, shift_x=0.05, energy="sg"),
}


@pytest.mark.parametrize("gamma", [4.0, 25.0])
@pytest.mark.parametrize("case", sorted(CASES))
def test_augmented_lagrangian_decreases_as_proposition_1_states(case, gamma):
    wl = CASES[case]()
    probe = admm.Oracle.from_workload(wl)
    s = probe.init(wl.W0)
    assert np.all(np.linalg.det(s.J) > 0)                     # an unflipped start (Sec. 6: h_i on)
    w, e = probe.w, probe.energy_name
    B = np.sqrt(5.0 * (1.0 + _gnorm(s.P, e) ** 2))            # Condition 1's bound as Sec. 6 sets it
    eps = 0.25 * w.min()                                       # 0 < eps < min w / 2
    F = schedule.lipschitz_F(B, e, probe.d)                    # Lemma 1
    a = w - 2.0 * eps
    mu = 1.0001 * 0.5 * (-a + np.sqrt(a * a + 16.0 * gamma * w * w * F * F))
    h = 4.0 * gamma * w * w * B * B / mu + 2.0 * eps
    o = admm.Oracle(wl.V, wl.T, wl.pins, wl.pin_pos, wl.energy, rho=1.0, h=h)
    schedule.set_penalties(o, mu)
    free = np.setdiff1d(np.arange(o.n), wl.pins)
    L = admm.assemble_L(o.g, o.T, o.mu, o.n)
    lam_min = np.linalg.eigvalsh(L[free][:, free].toarray())[0]
    assert lam_min > 0
    tr = lambda X: np.transpose(X, (0, 2, 1))
    s = o.init(wl.W0)
    applied = 0
    for k in range(60):
        s1, _ = o.step(s)
        # from k = 1 on: P^k then comes from a P step, whose optimality the proof uses
        if k >= 1:
            c1 = np.all(_gnorm(s.P, e) <= B) and np.all(_gnorm(s1.P, e) <= B)
            D = s1.Lam - s.Lam
            S = s1.Lam + s1.U @ tr(s1.Lam) @ s1.U - s.Lam - s.U @ tr(s.Lam) @ s.U
            c2 = np.all(np.einsum("mij,mij->m", D, D) <= gamma / 4.0 * np.einsum("mij,mij->m", S, S))
            if c1 and c2:
                applied += 1
                lhs = _phi(o, s1) - _phi(o, s)
                rhs = (-0.5 * lam_min * np.sum((s1.W - s.W) ** 2)
                       - eps * (np.sum((s1.U - s.U) ** 2) + np.sum((s1.P - s.P) ** 2)))
                assert lhs <= rhs + 1e-12 * (1.0 + abs(_phi(o, s))), (k, lhs, rhs)
        s = s1
    # the proposition applied on most steps (it says nothing where a condition fails)
    assert applied >= 25, applied
