"""The oracle against the convergence behaviour the paper reports (Fig. 3, with
Sec. 5, Conditions 1 and 2): on UV parametrizations the primal and dual errors
decrease steadily, while the largest gradient |grad f(P_i)| (a proxy for the
bound B_i of Condition 1) and the largest Lambda ratio (a proxy for gamma^{1/2}
of Condition 2) stay bounded.  The Lambda ratio itself is first pinned on states
written out by hand.  No GPU is used."""
import math

import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def _tiny_oracle(m):
    """An oracle whose mesh only fixes m and mu (the proxies read the states given)."""
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])[:m + 2]
    T = np.array([[0, 1, 2], [1, 3, 2]])[:m]
    return admm.Oracle(V, T, np.array([0]), np.zeros((1, 2)), "sd", rho=3.0)


def _state(U, P, Lam):
    U, P, Lam = (np.asarray(x, float) for x in (U, P, Lam))
    return admm.State(np.zeros((4, 2)), U, P, Lam, np.zeros_like(Lam))


def test_lambda_ratio_by_hand():
    o = _tiny_oracle(1)
    I = np.eye(2)[None]
    Z = np.zeros((1, 2, 2))
    c, s = math.cos(0.7), math.sin(0.7)
    R = np.array([[[c, -s], [s, c]]])
    Sym = np.array([[[2.0, 1.0], [1.0, -3.0]]])
    Anti = np.array([[[0.0, 1.5], [-1.5, 0.0]]])
    # a symmetric multiplier step with U = I: the bracket is the step itself, ratio 1
    _, r = o.condition_proxies(_state(I, I, Z), _state(I, I, Sym))
    assert math.isclose(r, 1.0, rel_tol=1e-14)
    # Lambda^{k+1} = R S with S symmetric and U^{k+1} = R: U M^T U = R S R^T R = R S,
    # so the bracket is again the step, ratio 1
    _, r = o.condition_proxies(_state(I, I, Z), _state(R, I, R @ Sym))
    assert math.isclose(r, 1.0, rel_tol=1e-12)
    # an antisymmetric step with U = I: the bracket vanishes, no gamma bounds it
    _, r = o.condition_proxies(_state(I, I, Z), _state(I, I, Anti))
    assert r == math.inf
    # symmetric plus antisymmetric, U = I: |S + A| / |S| = sqrt(|S|^2 + |A|^2) / |S|
    _, r = o.condition_proxies(_state(I, I, Z), _state(I, I, Sym + Anti))
    want = math.sqrt(np.sum(Sym ** 2) + np.sum(Anti ** 2)) / math.sqrt(np.sum(Sym ** 2))
    assert math.isclose(r, want, rel_tol=1e-14)
    # the multiplier is mu Lambda, with each state's own penalty: mu0 = 1, mu1 = 2
    # and Lambda^k = Sym / 2 give M^k = Sym / 2, M^{k+1} = 2 Sym, a symmetric step
    # (ratio 1); a state that did not move is skipped
    _, r = o.condition_proxies(_state(I, I, Sym / 2), _state(I, I, Sym), mu0=[1.0], mu1=[2.0])
    assert math.isclose(r, 1.0, rel_tol=1e-14)
    _, r = o.condition_proxies(_state(I, I, Sym), _state(I, I, Sym))
    assert r == 0.0
    # where the scaling does not cancel: Lambda^k = A, Lambda^{k+1} = A + S, U = I,
    # mu0 = 1, mu1 = 2: M^k = A, M^{k+1} = 2A + 2S, D = A + 2S, and the bracket is
    # (D + M^{k+1 T} - M^{k T}) / 2 = (A + 2S - 2A + 2S + A) / 2 = 2S, so the ratio is
    # sqrt(|A|^2 + 4|S|^2) / (2|S|); with the scaled Lambda alone it would be 1
    _, r = o.condition_proxies(_state(I, I, Anti), _state(I, I, Anti + Sym), mu0=[1.0], mu1=[2.0])
    want = math.sqrt(np.sum(Anti ** 2) + 4 * np.sum(Sym ** 2)) / (2 * math.sqrt(np.sum(Sym ** 2)))
    assert math.isclose(r, want, rel_tol=1e-14) and not math.isclose(r, 1.0)
    # the gradient proxy: |grad f_SD(pI)| = sqrt(2) |p - p^-3| in 2D
    g, _ = o.condition_proxies(_state(I, I, Z), _state(I, 2.0 * I, Z))
    assert math.isclose(g, math.sqrt(2.0) * (2.0 - 2.0 ** -3), rel_tol=1e-14)


def _dyadic_maxima(vals, start):
    """max of vals[k] over k in [2^j, 2^{j+1}) (k counted from 1), for 2^j >= start."""
    out = []
    j = 0
    while 2 ** j <= len(vals):
        lo, hi = 2 ** j, min(2 ** (j + 1), len(vals) + 1)
        if lo >= start:
            out.append(max(vals[lo - 1:hi - 1]))
        j += 1
    return out


@pytest.mark.parametrize("name", ["disk_sd", "heightfield_sg"])
def test_errors_decrease_and_the_condition_proxies_stay_bounded(name):
    if name == "disk_sd":
        wl = wk.uv_disk(grid=24, rho=3.0)
    else:
        wl = wk.uv_heightfield(grid=24, rho=10.0)
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    ep, ed, gs, rs = [], [], [], []
    for _ in range(200):
        s1, st = o.step(s)
        g, r = o.condition_proxies(s, s1)
        ep.append(st.e_prim)
        ed.append(st.e_dual)
        gs.append(g)
        rs.append(r)
        s = s1
        if st.converged:
            break
    assert st.converged and st.n_flipped == 0
    # the errors decrease steadily: their maxima over dyadic windows of iterations
    # fall from window to window (e_dual after its first iteration, where it starts
    # from the polar initialization's J^0), by three orders of magnitude overall
    mp, md = _dyadic_maxima(ep, 1), _dyadic_maxima(ed, 2)
    assert all(b < a for a, b in zip(mp, mp[1:])), mp
    assert all(b < a for a, b in zip(md, md[1:])), md
    assert ep[-1] < 1e-3 * ep[0]
    # the proxies stay bounded: the gradient never exceeds twice its first value,
    # and the Lambda ratio stays finite, moderate, and ends near 1
    assert max(gs) <= 2.0 * gs[0], (gs[0], max(gs))
    assert all(math.isfinite(r) for r in rs) and max(rs) < 50.0
    assert rs[-1] < 2.0
