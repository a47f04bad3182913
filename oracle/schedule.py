"""FP64 CPU oracle of the paper's penalty schedule (Algorithm 2; Sec. 6,
"Rescaling mu_i and Lambda"; Lemma 1 and Proposition 1 of Sec. 5).

TEST INFRASTRUCTURE ONLY, like oracle/admm.py: only the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import it.

What it adds to the fixed-penalty loop of oracle/admm.py:
  * B_i = sqrt(5 (1 + |grad f(P_i)|^2))      (the bound of Condition 1, as Sec. 6 sets it)
  * F_i from Lemma 1: SG  F = 1 + sqrt(d) / (C^L)^2,   C^L the positive root of x^2 + B x - 1
                      SD  F = 1 + 3 sqrt(d) / (C^LG)^4, C^LG the positive root of x^4 + B x^3 - 1
    with F_i^2 capped at eps_m^(-1/4) (Sec. 6).
  * mu_min,i = (-(w_i - 2 eps) + sqrt((w_i - 2 eps)^2 + 16 gamma w_i^2 F_i^2)) / 2 with
    gamma = 1, eps = 0 (Proposition 1, values from Sec. 6).
  * initial penalties mu_i = max(mu_min,i(P^0), w_i) (Algorithm 2).
  * rescaling (Sec. 6): if e_prim_i > rho e_dual_i then mu_i *= rho/2, if
    e_dual_i > rho e_prim_i then mu_i /= rho/2, rho = 5, never below
    mu_min,i(P^k) / 2; the scaled multiplier follows so that mu_i Lambda_i is
    unchanged.
  * the events: five times directly after initialization (after iterations
    1..5), then after every floor(5 (3/2)^p) iterations, p the number of past
    events; L is decomposed again after each event.

Readings (also in the design notes): C^L = (-B + sqrt(4 + B^2))/2 is evaluated as
the equal 2 / (B + sqrt(4 + B^2)), which does not cancel for large B; the
Lambda factor is mu_old/mu_new, which
is the printed "divide/multiply by rho/2" whenever the lower bound does not
bind; the termination test of an event iteration is evaluated on that
iteration's iterate before its rescaling (Algorithm 2 lists the test after the
rescaling; testing first lets a converged iterate stop without a needless
decomposition of L); an element error below 2^-40 (1 + |J_i|) (times mu_i for
e_dual) counts as zero, so that elements that have stopped moving are not
rescaled on rounding noise (the paper's rule leaves both errors exactly zero
alone); h_i = 0 as in the fixed-penalty loop.
"""
from __future__ import annotations

import math

import numpy as np

from . import admm

RESCALE_RHO = 5.0
F2_CAP = admm.EPS_M ** -0.25


def grad_f_norm(P: np.ndarray, energy_name: str) -> np.ndarray:
    """|grad f(P_i)| (Frobenius) from the closed-form gradients of oracle/admm.py."""
    G = admm.grad_f(P, energy_name)
    return np.sqrt(np.einsum("mij,mij->m", G, G))


def c_lipschitz(B: np.ndarray, energy_name: str) -> np.ndarray:
    """C^L (SG, closed form) or C^LG (SD, bisection to adjacent doubles) of Lemma 1."""
    if energy_name not in ("sd", "sg"):
        raise ValueError("Lemma 1 bounds the Lipschitz constant for the SD and SG energies only")
    if energy_name == "sg":
        # (-B + sqrt(4 + B^2)) / 2, written without the cancellation for large B
        return 2.0 / (B + np.sqrt(4.0 + B * B))
    # x^4 + B x^3 - 1 is -1 at 0 and B >= 0 at 1 and increasing on [0, 1]
    lo = np.zeros_like(B)
    hi = np.ones_like(B)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        neg = mid ** 4 + B * mid ** 3 - 1.0 < 0.0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
        if np.all(np.nextafter(lo, np.inf) >= hi):
            break
    return 0.5 * (lo + hi)


def lipschitz_F(B: np.ndarray, energy_name: str, d: int) -> np.ndarray:
    """F_i of Lemma 1, with F_i^2 capped at eps_m^(-1/4) (Sec. 6)."""
    C = c_lipschitz(B, energy_name)
    F = 1.0 + math.sqrt(d) / C ** 2 if energy_name == "sg" else 1.0 + 3.0 * math.sqrt(d) / C ** 4
    return np.minimum(F, math.sqrt(F2_CAP))


def mu_min(P: np.ndarray, w: np.ndarray, energy_name: str) -> np.ndarray:
    """mu_min,i of Proposition 1 with gamma = 1, eps = 0 and B_i from P_i (Sec. 6)."""
    d = P.shape[1]
    B = np.sqrt(5.0 * (1.0 + grad_f_norm(P, energy_name) ** 2))
    F = lipschitz_F(B, energy_name, d)
    return 0.5 * (-w + np.sqrt(w * w + 16.0 * w * w * F * F))


def h_bound(P: np.ndarray, w: np.ndarray, mu: np.ndarray, energy_name: str) -> np.ndarray:
    """The proximal weight of eq. proximalfunctionu at the bound of Proposition 1,
    h_i = 4 gamma w_i^2 B_i^2 / mu_i + 2 eps with gamma = 1, eps = 0 (Sec. 6: "h_i is set to
    its value from" the convergence section), B_i = sqrt(5 (1 + |grad f(P_i)|^2)) as for mu_min."""
    B2 = 5.0 * (1.0 + grad_f_norm(P, energy_name) ** 2)
    return 4.0 * w * w * B2 / mu


def rescale(mu, Lam, e_prim_i, e_dual_i, mu_lo, rho: float = RESCALE_RHO):
    """One rescaling of every element's penalty and scaled multiplier (Sec. 6)."""
    new = mu.copy()
    up = e_prim_i > rho * e_dual_i
    down = e_dual_i > rho * e_prim_i
    new[up] *= 0.5 * rho
    new[down] /= 0.5 * rho
    new = np.maximum(new, mu_lo)
    return new, Lam * (mu / new)[:, None, None]


def rescale_iterations(max_iter: int) -> list[int]:
    """Iterations after which Algorithm 2 rescales: 1..5, then every floor(5 (3/2)^p)."""
    ev = [k for k in range(1, 6) if k <= max_iter]
    k, p = 5, 5
    while True:
        k += int(math.floor(5.0 * 1.5 ** p))
        if k > max_iter:
            return ev
        ev.append(k)
        p += 1


ROUNDING_FLOOR = 2.0 ** -40


def element_errors(o: admm.Oracle, s0: admm.State, s1: admm.State):
    """e_prim_i and e_dual_i of eq. primaldualerror for every element; an error
    below the rounding floor of its element (2^-40 (1 + |J_i|), times mu_i for
    e_dual) counts as zero."""
    R = s1.J - s1.U @ s1.P
    D = s1.J - s0.J
    ep = np.sqrt(np.einsum("mij,mij->m", R, R))
    ed = o.mu * np.sqrt(np.einsum("mij,mij->m", D, D))
    floor = ROUNDING_FLOOR * (1.0 + np.sqrt(np.einsum("mij,mij->m", s1.J, s1.J)))
    return np.where(ep > floor, ep, 0.0), np.where(ed > o.mu * floor, ed, 0.0)


def set_penalties(o: admm.Oracle, mu: np.ndarray) -> None:
    """New penalties: decompose L again (Algorithm 2, decompose(L))."""
    o.mu = np.asarray(mu, np.float64).copy()
    o.wstep = admm.WStep(o.g, o.T, o.mu, o.n, o.wstep.pins, o.wstep.pin_pos)


def run(o: admm.Oracle, W0, max_iter: int, stop_at_tol: bool = True, callback=None):
    """Algorithm 2 with the rescaling branch.  Returns the last state, its stats
    and the number of rescaling events."""
    s = o.init(W0)
    set_penalties(o, np.maximum(mu_min(s.P, o.w, o.energy_name), o.w))
    events = set(rescale_iterations(max_iter))
    st, n_events = None, 0
    for k in range(1, max_iter + 1):
        W = o.w_step(s)
        s1 = o.local_steps(s, W)
        st = o.stats(s, s1, k)
        if callback is not None:
            callback(k, s, s1, st)
        if stop_at_tol and st.converged:
            return s1, st, n_events
        if k in events:
            ep, ed = element_errors(o, s, s1)
            mu_new, s1.Lam = rescale(o.mu, s1.Lam, ep, ed, 0.5 * mu_min(s1.P, o.w, o.energy_name))
            set_penalties(o, mu_new)
            n_events += 1
        s = s1
    return s, st, n_events
