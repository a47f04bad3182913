"""Pins of the oracle's termination quantities (Sec. 6, "Termination Condition":
eqs. primaldualerror and primaldualthresholds) against values worked out by hand.

The mesh is the unit square split into two triangles,
    V = (0,0), (1,0), (0,1), (1,1);   T = [0,1,2], [1,3,2];   w_0 = w_1 = 1/2,
so d = 2, m = 2 and, with rho = 3, mu_0 = mu_1 = 3/2.  The hat-function gradients
(row j = gradient of the hat function of T_ij) are, by hand,
    element 0: v0 (-1,-1), v1 (1,0), v2 (0,1)
    element 1: v1 (0,-1), v3 (1,1), v2 (-1,0).
The states are written out entry by entry (they need not come from an iteration:
the formulas are evaluated on whatever state they are given).  Every expected
number below is a sum of squares done by hand, with the arithmetic in the
comment beside it; nothing is recomputed with the oracle's own helpers.  Each
case is built so that one plausible misreading changes the result:
sqrt(d^2 m) or sqrt(m) for sqrt(d m), mu_i for mu_i^2, |U P| for |P|, |J| alone
for the max, G^T (mu Lambda) or a transposed Lambda_i in G^T Lambda, det J < 0
for det J <= 0 as the flip test.
"""
import math

import numpy as np

from oracle import admm

V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
T = np.array([[0, 1, 2], [1, 3, 2]])


def _oracle(eps_abs, eps_rel, energy="sd"):
    return admm.Oracle(V, T, np.array([0]), np.zeros((1, 2)), energy, rho=3.0,
                       eps_abs=eps_abs, eps_rel=eps_rel)


def _state(J, U, P, Lam):
    J = np.asarray(J, float)
    return admm.State(np.zeros((4, 2)), np.asarray(U, float), np.asarray(P, float),
                      np.asarray(Lam, float), J)


I2 = np.eye(2)


def test_hat_gradients_are_the_ones_worked_by_hand():
    o = _oracle(1e-6, 1e-5)
    np.testing.assert_allclose(o.g[0], [[-1, -1], [1, 0], [0, 1]], atol=1e-15)
    np.testing.assert_allclose(o.g[1], [[0, -1], [1, 1], [-1, 0]], atol=1e-15)
    np.testing.assert_allclose(o.w, [0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(o.mu, [1.5, 1.5], atol=1e-15)


def test_errors_and_thresholds_case_a():
    """A state whose thresholds are set by |P| and by G^T Lambda with a non-symmetric Lambda_1."""
    o = _oracle(eps_abs=0.1, eps_rel=0.01)
    s0 = _state([I2, I2], [I2, I2], [I2, I2], [np.zeros((2, 2))] * 2)
    J1 = [[[1.2, 0.0], [0.0, 1.0]], [[1.0, 0.1], [0.0, 1.0]]]
    P1 = [I2, [[1.0, 0.0], [0.0, 2.0]]]
    Lam1 = [[[1.0, 0.0], [0.0, 0.0]], [[0.0, 1.0], [0.0, 2.0]]]
    s1 = _state(J1, [I2, I2], P1, Lam1)
    st = o.stats(s0, s1)
    # J - U P: element 0 [[0.2,0],[0,0]] -> 0.04; element 1 [[0,0.1],[0,-1]] -> 0.01 + 1
    assert math.isclose(st.e_prim, math.sqrt(1.05), rel_tol=1e-14)
    # J^k - J^(k-1): 0.04 and 0.01; times mu^2 = 2.25: 2.25 * 0.05 = 0.1125
    assert math.isclose(st.e_dual, math.sqrt(0.1125), rel_tol=1e-14)
    # eps_abs sqrt(d m) = 0.1 * sqrt(4) = 0.2
    # |J|^2 = (1.44 + 1) + (1 + 0.01 + 1) = 4.45 ; |P|^2 = 2 + (1 + 4) = 7 -> max is sqrt 7
    assert math.isclose(st.thr_prim, 0.2 + 0.01 * math.sqrt(7.0), rel_tol=1e-14)
    # G^T Lambda, by hand (column k of Lambda_i dotted with each hat gradient):
    #   element 0, column 0 = (1,0): v0 -1, v1 +1, v2 0 (column 1 is zero)
    #   element 1, column 1 = (1,2): v1 (0,-1).(1,2) = -2, v3 (1,1).(1,2) = 3, v2 (-1,0).(1,2) = -1
    #   rows: v0 (-1,0), v1 (1,-2), v2 (0,-1), v3 (0,3) -> |G^T Lambda|^2 = 1+1+4+1+9 = 16
    assert math.isclose(st.thr_dual, 0.2 + 0.01 * 4.0, rel_tol=1e-14)
    assert st.n_flipped == 0
    # SD: f(P) = (|P|^2 + |P^-1|^2)/2 ; element 0: (2 + 2)/2 = 2 ; element 1: (5 + 1.25)/2 = 3.125
    assert math.isclose(st.energy_P, 0.5 * 2.0 + 0.5 * 3.125, rel_tol=1e-14)
    assert not st.converged


def test_errors_and_thresholds_case_b():
    """|J| above |P| sets the primal threshold; |U P| would differ from |P| (U = 2I here is not
    a rotation, which only a hand-made state can have); det J = 0 counts as flipped."""
    o = _oracle(eps_abs=1.0, eps_rel=0.1)
    J = [[[3.0, 0.0], [0.0, 1.0]], [[1.0, 0.0], [0.0, 0.0]]]
    U = [2.0 * I2, I2]
    P = [[[1.5, 0.0], [0.0, 0.5]], [[1.0, 0.0], [0.0, 0.5]]]
    s = _state(J, U, P, [np.zeros((2, 2))] * 2)
    st = o.stats(s, s)
    # J - U P: element 0: [[3,0],[0,1]] - [[3,0],[0,1]] = 0 ; element 1: [[0,0],[0,-0.5]] -> 0.25
    assert math.isclose(st.e_prim, 0.5, rel_tol=1e-14)
    assert st.e_dual == 0.0
    # |J|^2 = 9 + 1 + 1 = 11 ; |P|^2 = 2.25 + 0.25 + 1 + 0.25 = 3.75 (|U P|^2 would be 11.25)
    # eps_abs sqrt(d m) = 1 * 2
    assert math.isclose(st.thr_prim, 2.0 + 0.1 * math.sqrt(11.0), rel_tol=1e-14)
    assert math.isclose(st.thr_dual, 2.0, rel_tol=1e-14)
    assert st.n_flipped == 1
    assert not st.converged           # both errors are below their thresholds, one element is flipped


def test_errors_and_thresholds_case_c_converges():
    """The same as case b with element 1 no longer degenerate: the test passes."""
    o = _oracle(eps_abs=1.0, eps_rel=0.1)
    J = [[[3.0, 0.0], [0.0, 1.0]], [[1.0, 0.0], [0.0, 0.25]]]
    U = [2.0 * I2, I2]
    P = [[[1.5, 0.0], [0.0, 0.5]], [[1.0, 0.0], [0.0, 0.5]]]
    st = o.stats(_state(J, U, P, [np.zeros((2, 2))] * 2), _state(J, U, P, [np.zeros((2, 2))] * 2))
    # J - U P, element 1: [[0,0],[0,-0.25]] -> e_prim = 0.25
    assert math.isclose(st.e_prim, 0.25, rel_tol=1e-14)
    # |J|^2 = 9 + 1 + 1 + 0.0625 = 11.0625
    assert math.isclose(st.thr_prim, 2.0 + 0.1 * math.sqrt(11.0625), rel_tol=1e-14)
    assert st.n_flipped == 0 and st.converged


def test_dual_error_uses_the_squared_penalty_per_element():
    """Different mu_i per element: e_dual^2 = sum_i mu_i^2 |dJ_i|^2 (eq. primaldualerror), not
    mu_i^2 summed separately from the differences."""
    o = _oracle(eps_abs=0.1, eps_rel=0.01)
    o.mu = np.array([1.0, 4.0])
    s0 = _state([I2, I2], [I2, I2], [I2, I2], [np.zeros((2, 2))] * 2)
    s1 = _state([[[1.0, 0.5], [0.0, 1.0]], [[1.0, 0.0], [0.25, 1.0]]], [I2, I2], [I2, I2],
                [np.zeros((2, 2))] * 2)
    st = o.stats(s0, s1)
    # 1^2 * 0.25 + 4^2 * 0.0625 = 0.25 + 1 = 1.25
    assert math.isclose(st.e_dual, math.sqrt(1.25), rel_tol=1e-14)


def test_threshold_base_in_3d_is_eps_abs_sqrt_d_m():
    """d = 3, m = 6 (one Kuhn-split cube): eps_abs sqrt(d m) = sqrt(18) with eps_abs = 1 and
    eps_rel = 0 (J = 0, U = P = I, Lambda = 0 in a hand state)."""
    from paper_2107_05200_gb300 import workloads as wk
    V3, T3 = wk.cube_tets(1)
    o = admm.Oracle(V3, T3, np.array([0]), np.zeros((1, 3)), "sd", eps_abs=1.0, eps_rel=0.0)
    Z = np.zeros((6, 3, 3))
    I3 = np.broadcast_to(np.eye(3), Z.shape).copy()
    s = admm.State(np.zeros((8, 3)), I3, I3, Z, Z)
    st = o.stats(s, s)
    assert math.isclose(st.thr_prim, math.sqrt(18.0), rel_tol=1e-14)
    assert math.isclose(st.thr_dual, math.sqrt(18.0), rel_tol=1e-14)
    assert st.n_flipped == 6          # det 0 <= 0 for all six


def test_flipped_polar_init_maximizes_the_trace_over_reflections():
    """Sec. 6, eq. polardecompositionapplied, checked by a property rather than by the formula:
    for det J < 0 the returned U is a rotation and U D (D = diag(1, .., 1, -1)) is the
    reflection nearest to J, i.e. it maximizes tr(O^T J) over orthogonal O with det O = -1
    (found here by an angle grid in 2D and a search over random rotations times D in 3D)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(21)
    for d in (2, 3):
        J = rng.normal(size=(30, d, d))
        J[np.linalg.det(J) > 0, :, 0] *= -1.0          # make every J flipped
        assert np.all(np.linalg.det(J) < 0)
        U, _ = admm.polar_init(J, "sd")
        D = np.diag([1.0] * (d - 1) + [-1.0])
        if d == 2:
            phi = np.linspace(0, 2 * math.pi, 400001)
            cands = np.stack([np.stack([np.cos(phi), np.sin(phi)], 1),
                              np.stack([np.sin(phi), -np.cos(phi)], 1)], 1)   # reflections
        else:
            cands = Rotation.random(200000, random_state=22).as_matrix() @ D
        for i in range(len(J)):
            assert math.isclose(np.linalg.det(U[i]), 1.0, rel_tol=1e-12)
            mine = np.trace((U[i] @ D).T @ J[i])
            best = np.max(np.einsum("cij,ij->c", cands, J[i]))
            assert mine >= best - 1e-9
            # det J < 0: the nearest reflection attains the sum of the singular values
            s = np.linalg.svd(J[i], compute_uv=False)
            assert math.isclose(mine, s.sum(), rel_tol=1e-12, abs_tol=1e-12)
