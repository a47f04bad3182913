"""Pins of the oracle's W step with general linear constraints A W = b (Sec. 4,
W update: any feasible A W = b; an indefinite system the paper hands to
UMFPACK): the KKT solve against the pinned elimination it generalizes, against a
dense null-space minimization, its feasibility, its refusal of constraints that
leave W's translations free, and a whole run held to a centroid constraint."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def _setup(wl, rho=3.0):
    T = wl.T.astype(np.int64)
    g, w = admm.element_gradients(wl.V, T)
    return T, g, rho * w, wl.V.shape[0]


@pytest.mark.parametrize("make", [lambda: wk.uv_disk(grid=9, seed=41), lambda: wk.cube_deform(cells=3, seed=42)])
def test_pins_as_constraints_equal_the_pinned_elimination(make):
    wl = make()
    T, g, mu, n = _setup(wl)
    rng = np.random.default_rng(1)
    rhs = rng.normal(size=(n, wl.V.shape[1]))
    W_elim = admm.WStep(g, T, mu, n, wl.pins, wl.pin_pos).solve(rhs)
    W_kkt = admm.WStepKKT(g, T, mu, n, admm.pin_rows(wl.pins, n), wl.pin_pos).solve(rhs)
    np.testing.assert_allclose(W_kkt, W_elim, rtol=0, atol=1e-12 * np.abs(W_elim).max())


def _general_constraints(n, d, rng):
    """Two pins, the centroid of five vertices, and a rigid link W_a = W_b."""
    rows, b = [], []
    for v in (0, 1):
        r = np.zeros(n)
        r[v] = 1.0
        rows.append(r)
        b.append(rng.normal(size=d))
    r = np.zeros(n)
    r[[3, 4, 5, 6, 7]] = 0.2
    rows.append(r)
    b.append(rng.normal(size=d))
    r = np.zeros(n)
    r[9], r[11] = 1.0, -1.0
    rows.append(r)
    b.append(np.zeros(d))
    return sp.csr_matrix(np.array(rows)), np.array(b)


@pytest.mark.parametrize("make", [lambda: wk.uv_disk(grid=7, seed=43), lambda: wk.cube_deform(cells=2, seed=44)])
def test_general_constraints_against_a_dense_null_space_minimization(make):
    """min 1/2 tr(W^T L W) - tr(rhs^T W) subject to A W = b, per coordinate column:
    W = W_p + N y with A W_p = b and N spanning null(A), (N^T L N) y = N^T (rhs - L W_p)."""
    wl = make()
    T, g, mu, n = _setup(wl)
    d = wl.V.shape[1]
    rng = np.random.default_rng(2)
    A, b = _general_constraints(n, d, rng)
    rhs = rng.normal(size=(n, d))
    W = admm.WStepKKT(g, T, mu, n, A, b).solve(rhs)
    Ad = A.toarray()
    L = admm.assemble_L(g, T, mu, n).toarray()
    Wp = np.linalg.lstsq(Ad, b, rcond=None)[0]
    N = sl.null_space(Ad)
    y = np.linalg.solve(N.T @ L @ N, N.T @ (rhs - L @ Wp))
    W_ref = Wp + N @ y
    np.testing.assert_allclose(A @ W, b, rtol=0, atol=1e-12)
    np.testing.assert_allclose(W, W_ref, rtol=0, atol=1e-10 * np.abs(W_ref).max())
    # stationarity: L W - rhs lies in the row space of A
    res = L @ W - rhs
    nu = np.linalg.lstsq(Ad.T, -res, rcond=None)[0]
    np.testing.assert_allclose(Ad.T @ nu, -res, rtol=0, atol=1e-9 * max(1.0, np.abs(res).max()))


def test_constraints_that_leave_translations_free_are_refused():
    wl = wk.uv_disk(grid=6, seed=45)
    T, g, mu, n = _setup(wl)
    r = np.zeros((1, n))
    r[0, 2], r[0, 3] = 1.0, -1.0   # W_2 = W_3 fixes no translation
    with pytest.raises(ValueError, match="translation"):
        admm.WStepKKT(g, T, mu, n, sp.csr_matrix(r), np.zeros((1, 2)))
    # the same vertex pinned twice: dependent rows
    with pytest.raises(ValueError, match="dependent"):
        admm.WStepKKT(g, T, mu, n, admm.pin_rows([4, 4], n), np.zeros((2, 2)))


def test_run_held_to_a_centroid_constraint():
    """The cube with its bottom face pinned and, instead of pinning every top-face
    vertex, only the top face's centroid moved: every iterate satisfies A W = b,
    and the iteration converges without flips."""
    wl = wk.cube_deform(cells=3, seed=46, angle_deg=0.0, shift_x=0.2)
    n = wl.V.shape[0]
    z = wl.V[:, 2]
    bottom = np.nonzero(z < 1e-9)[0]
    top = np.nonzero(z > 1 - 1e-9)[0]
    A = sp.csr_matrix((np.full(len(top), 1.0 / len(top)), (np.zeros(len(top), int), top)), shape=(1, n))
    b = (wl.V[top].mean(axis=0) + np.array([0.2, 0.0, 0.1]))[None]
    o = admm.Oracle(wl.V, wl.T, bottom, wl.V[bottom], wl.energy, rho=3.0, constraints=(A, b))
    W0 = wl.V.copy()
    W0[top] += np.array([0.2, 0.0, 0.1])
    seen = []

    def cb(k, s0, s1, st):
        np.testing.assert_allclose(A @ s1.W, b, rtol=0, atol=1e-12)
        np.testing.assert_allclose(s1.W[bottom], wl.V[bottom], rtol=0, atol=1e-12)
        seen.append(st)

    s, st = o.run(W0, 400, callback=cb)
    assert st.converged and st.n_flipped == 0, (st.k, st.e_prim, st.thr_prim)
    assert seen[-1].e_prim < 1e-3 * max(seen[0].e_prim, 1e-30)
