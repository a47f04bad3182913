"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
brute-force minimization on tiny inputs, adjointness and quadratic-form
identities, invariants (rigid motions, KKT conditions) and the convergence
behaviour the paper reports.  No GPU is used.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so
from scipy.spatial.transform import Rotation

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def _small_meshes():
    V2, T2 = wk.grid_triangles(5, 4)
    rng = np.random.default_rng(0)
    V2 = V2 + rng.uniform(-0.03, 0.03, V2.shape)
    V3, T3 = wk.cube_tets(2)
    V3 = V3 + rng.uniform(-0.03, 0.03, V3.shape)
    # a planar patch rotated into R^3: an intrinsic (surface) mesh
    R = Rotation.from_rotvec([0.3, -0.7, 0.2]).as_matrix()
    Vs = np.column_stack([V2, np.zeros(len(V2))]) @ R.T + np.array([0.1, 0.2, 0.3])
    return [(V2, T2), (V3, T3), (Vs, T2)]


# --------------------------------------------------------------------------
# mesh operators
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 1])
def test_affine_maps_reproduce_their_matrix(k):
    """Def. jacobian (Sec. 3.1) + Supplemental: for W = V M + t every J_i equals M (column k = grad W_k)."""
    V, T = _small_meshes()[k]
    g, w = admm.element_gradients(V, T)
    rng = np.random.default_rng(1)
    d = V.shape[1]
    M = rng.normal(size=(d, d))
    W = V @ M + rng.normal(size=d)
    J = admm.jacobians(g, T, W)
    np.testing.assert_allclose(J, np.broadcast_to(M, J.shape), atol=1e-11)


def test_intrinsic_jacobian_of_isometry_is_rotation():
    """Surface triangles: an isometric flattening has J in SO(2) in the intrinsic frame."""
    V2, T2 = _small_meshes()[0]
    Vs = _small_meshes()[2][0]
    g, w = admm.element_gradients(Vs, T2)
    J = admm.jacobians(g, T2, V2)          # flatten back to the original plane
    np.testing.assert_allclose(np.einsum("mji,mjk->mik", J, J), np.broadcast_to(np.eye(2), J.shape), atol=1e-11)
    np.testing.assert_allclose(np.linalg.det(J), 1.0, atol=1e-11)
    g2, w2 = admm.element_gradients(V2, T2)
    np.testing.assert_allclose(w, w2, rtol=1e-12)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_constants_are_annihilated(k):
    """Sec. 4 (W update): G maps constant functions to zero."""
    V, T = _small_meshes()[k]
    g, _ = admm.element_gradients(V, T)
    d = T.shape[1] - 1
    W = np.tile(np.arange(1.0, d + 1), (V.shape[0], 1))
    assert np.abs(admm.jacobians(g, T, W)).max() < 1e-12


def test_element_measures_sum_to_domain():
    """w_i are areas / volumes: they tile the unit square and the unit cube."""
    V, T = wk.grid_triangles(7, 5)
    assert math.isclose(admm.element_gradients(V, T)[1].sum(), 1.0, rel_tol=1e-13)
    V, T = wk.cube_tets(3)
    assert math.isclose(admm.element_gradients(V, T)[1].sum(), 1.0, rel_tol=1e-13)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_adjoint_and_quadratic_form(k):
    """<GW, R> = <W, G^T R>, and sum_i mu_i |(GW)_i|^2 = sum_k W_k^T L W_k (eq. solvinginw)."""
    V, T = _small_meshes()[k]
    g, w = admm.element_gradients(V, T)
    rng = np.random.default_rng(2)
    d = T.shape[1] - 1
    W = rng.normal(size=(V.shape[0], d))
    R = rng.normal(size=(T.shape[0], d, d))
    lhs = np.sum(admm.jacobians(g, T, W) * R)
    rhs = np.sum(W * admm.gradient_adjoint(g, T, R, V.shape[0]))
    assert math.isclose(lhs, rhs, rel_tol=1e-12)
    mu = rng.uniform(0.5, 2.0, size=T.shape[0]) * w
    J = admm.jacobians(g, T, W)
    L = admm.assemble_L(g, T, mu, V.shape[0])
    q1 = np.sum(mu[:, None, None] * J * J)
    q2 = sum(W[:, c] @ (L @ W[:, c]) for c in range(d))
    assert math.isclose(q1, q2, rel_tol=1e-12)


# --------------------------------------------------------------------------
# defining functions
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_energy_closed_forms_and_rotation_invariance(d):
    """f_SD(sI) = d(s^2+s^-2)/2, f_SG(sI) = d s^2/2 - d log s; f(RX) = f(X) (eqs. symmetricgradientdefiningfunction, symmetricdirichletdefiningfunction)."""
    s = 1.7
    X = (s * np.eye(d))[None]
    assert math.isclose(admm.f_energy(X, "sd")[0], d * (s * s + 1 / (s * s)) / 2, rel_tol=1e-14)
    assert math.isclose(admm.f_energy(X, "sg")[0], d * s * s / 2 - d * math.log(s), rel_tol=1e-14)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(5, d, d))
    A[np.linalg.det(A) < 0, :, 0] *= -1
    if d == 3:
        Rm = Rotation.random(5, random_state=4).as_matrix()
    else:
        phi = rng.uniform(0, 6, 5)
        Rm = admm.rot2(np.cos(phi), np.sin(phi))
    for e in ("sd", "sg"):
        np.testing.assert_allclose(admm.f_energy(Rm @ A, e), admm.f_energy(A, e), rtol=1e-12)


@pytest.mark.parametrize("energy", ["sd", "sg", "sa"])
def test_grad_f_matches_finite_differences(energy):
    """eq. symmetricgradientdefininggrad / eq. symmetricdirichletdefininggrad against central differences of f."""
    rng = np.random.default_rng(5)
    X = np.eye(3)[None] + 0.3 * rng.normal(size=(1, 3, 3))
    G = admm.grad_f(X, energy)[0]
    h = 1e-6
    for a in range(3):
        for b in range(3):
            E = np.zeros((1, 3, 3))
            E[0, a, b] = h
            fd = (admm.f_energy(X + E, energy)[0] - admm.f_energy(X - E, energy)[0]) / (2 * h)
            assert abs(fd - G[a, b]) < 1e-7 * max(1.0, abs(G[a, b]))


# --------------------------------------------------------------------------
# P step (eqs. optimizinginp/rootfindinginp, Supplemental eqs. genericpeqtosolve..peqfsdpluggedin)
# --------------------------------------------------------------------------

QS = [-100.0, -3.0, -1e-3, 0.0, 1e-9, 0.5, 1.0, 2.0, 50.0]
WM = [(1.0, 1.0), (1e-4, 1e-4), (1e-4, 3e-4), (2.0, 0.1), (0.1, 20.0)]


def _scalar_f(p, energy):
    if energy == "sa":
        return 0.5 * ((p - 1) ** 2 + (1 / p - 1) ** 2)
    return 0.5 * (p * p + 1 / (p * p)) if energy == "sd" else 0.5 * p * p - math.log(p)


@pytest.mark.parametrize("energy", ["sd", "sg", "sa"])
def test_scalar_prox_is_the_1d_minimizer(energy):
    """Each eigenvalue solves min_p w f(p) + mu/2 (p - q)^2 over p > 0 (brute force)."""
    root = {"sd": admm.root_sd, "sg": admm.root_sg, "sa": admm.root_sa}[energy]
    for (w, mu) in WM:
        q = np.array(QS)
        p = root(q, np.full_like(q, w), np.full_like(q, mu))
        for qi, pi in zip(QS, p):
            obj = lambda x: w * _scalar_f(x, energy) + 0.5 * mu * (x - qi) ** 2
            # bracket the minimizer on a log grid, then refine
            xs = np.exp(np.linspace(math.log(1e-6), math.log(200), 4001))
            j = int(np.argmin([obj(x) for x in xs]))
            res = so.minimize_scalar(obj, bounds=(xs[max(j - 1, 0)], xs[min(j + 1, len(xs) - 1)]),
                                     method="bounded", options=dict(xatol=1e-14))
            assert pi > 0
            assert abs(res.x - pi) <= 1e-6 * max(1.0, pi), (w, mu, qi, pi, res.x)
            assert obj(pi) <= obj(res.x) + 1e-12 * max(1.0, abs(obj(pi)))


@pytest.mark.parametrize("energy", ["sd", "sg", "sa"])
def test_scalar_prox_polynomial_residual(energy):
    """The root satisfies (w+mu)p^2 - mu q p - w = 0 (SG), (w+mu)p^4 - mu q p^3 - w = 0 (SD) or
    (w+mu)p^4 - (w + mu q)p^3 + w p - w = 0 (SA)."""
    rng = np.random.default_rng(6)
    q = rng.normal(scale=5, size=2000)
    w = rng.uniform(1e-5, 1.0, size=2000)
    mu = w * rng.uniform(0.5, 30, size=2000)
    if energy == "sd":
        p = admm.root_sd(q, w, mu)
        res = (w + mu) * p ** 4 - mu * q * p ** 3 - w
        scale = (w + mu) * p ** 4 + np.abs(mu * q * p ** 3) + w
    elif energy == "sa":
        # w phi'(p) + mu (p - q) = 0 with phi'(p) = p - 1 - p^-3 + p^-2, times p^3
        p = admm.root_sa(q, w, mu)
        res = (w + mu) * p ** 4 - (w + mu * q) * p ** 3 + w * p - w
        scale = (w + mu) * p ** 4 + np.abs((w + mu * q) * p ** 3) + w * p + w
    else:
        p = admm.root_sg(q, w, mu)
        res = (w + mu) * p ** 2 - mu * q * p - w
        scale = (w + mu) * p ** 2 + np.abs(mu * q * p) + w
    assert np.all(p > 0)
    assert np.max(np.abs(res) / scale) < 1e-13


def _spd_from_params(x, d):
    Lc = np.zeros((d, d))
    Lc[np.tril_indices(d)] = x
    Lc[np.diag_indices(d)] = np.exp(Lc[np.diag_indices(d)])
    return Lc @ Lc.T


@pytest.mark.parametrize("energy", ["sd", "sg", "sa"])
@pytest.mark.parametrize("d", [2, 3])
def test_matrix_prox_brute_force(energy, d):
    """P = argmin_{SPD} w f(P) + mu/2 |P - S|^2, found independently by BFGS over SPD matrices."""
    rng = np.random.default_rng(7 + d)
    for trial in range(4):
        A = rng.normal(size=(d, d))
        S = 0.5 * (A + A.T) * (0.5 + trial)
        w, mu = 0.7, [0.3, 1.0, 4.0, 0.05][trial]
        P = admm.p_step(S[None], np.array([w]), np.array([mu]), energy)[0]

        def obj(x):
            X = _spd_from_params(x, d)
            return w * admm.f_energy(X[None], energy)[0] + 0.5 * mu * np.sum((X - S) ** 2)

        best = None
        for start in range(3):
            x0 = rng.normal(scale=0.3, size=d * (d + 1) // 2)
            r = so.minimize(obj, x0, method="BFGS", options=dict(gtol=1e-11, maxiter=10000))
            if best is None or r.fun < best.fun:
                best = r
        Pb = _spd_from_params(best.x, d)
        assert np.all(np.linalg.eigvalsh(P) > 0)
        assert obj_val(P, S, w, mu, energy) <= best.fun + 1e-9
        np.testing.assert_allclose(P, Pb, atol=2e-4)


def obj_val(P, S, w, mu, energy):
    return w * admm.f_energy(P[None], energy)[0] + 0.5 * mu * np.sum((P - S) ** 2)


def test_eigenvalue_floor():
    """Supplemental: when det P or tr P < sqrt(eps_m), eigenvalues are raised to sqrt(eps_m)."""
    # a scalar problem whose SG root is ~1e-12: w tiny and q very negative
    S = np.diag([-1e6, 1.0])[None]
    P = admm.p_step(S, np.array([1e-12]), np.array([1.0]), "sg")[0]
    ev = np.linalg.eigvalsh(P)
    assert ev.min() == pytest.approx(admm.SQRT_EPS_M, rel=1e-12)


# --------------------------------------------------------------------------
# U step (eqs. rawoptimizationinudecoupled/optimizationinudecoupled, Supplemental)
# --------------------------------------------------------------------------

def test_procrustes_2d_against_angle_grid():
    rng = np.random.default_rng(8)
    Q = rng.normal(size=(50, 2, 2))
    U = admm.procrustes(Q, np.broadcast_to(np.eye(2), Q.shape).copy())
    phis = np.linspace(0, 2 * math.pi, 200001)
    Ug = admm.rot2(np.cos(phis), np.sin(phis))
    for i in range(len(Q)):
        obj = np.sum((Ug - Q[i]) ** 2, axis=(1, 2))
        best = obj.min()
        mine = np.sum((U[i] - Q[i]) ** 2)
        assert mine <= best + 1e-12
        assert abs(np.linalg.det(U[i]) - 1) < 1e-14


def test_procrustes_2d_tie_keeps_previous():
    Q = np.array([[[1.0, 2.0], [2.0, -1.0]]])      # q11+q22 = 0 and q21-q12 = 0
    Up = admm.rot2(np.array([0.6]), np.array([0.8]))
    np.testing.assert_array_equal(admm.procrustes(Q, Up.copy()), Up)


def test_procrustes_3d_against_rotation_search():
    rng = np.random.default_rng(9)
    Q = rng.normal(size=(12, 3, 3))
    Q[:4] = -Q[:4] if np.linalg.det(Q[0]) > 0 else Q[:4]   # include reflections
    U = admm.procrustes(Q, np.broadcast_to(np.eye(3), Q.shape).copy())
    Rs = Rotation.random(20000, random_state=10).as_matrix()
    for i in range(len(Q)):
        obj = np.sum((Rs - Q[i]) ** 2, axis=(1, 2))
        x0 = Rotation.from_matrix(Rs[int(np.argmin(obj))]).as_rotvec()
        f = lambda v: np.sum((Rotation.from_rotvec(v).as_matrix() - Q[i]) ** 2)
        r = so.minimize(f, x0, method="Nelder-Mead", options=dict(xatol=1e-12, fatol=1e-14, maxiter=20000))
        mine = np.sum((U[i] - Q[i]) ** 2)
        assert mine <= r.fun + 1e-9
        np.testing.assert_allclose(U[i].T @ U[i], np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(U[i]) - 1) < 1e-13


# --------------------------------------------------------------------------
# initialization (eqs. initialpolardecomposition/polardecompositionapplied)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_polar_init(d):
    rng = np.random.default_rng(11)
    J = rng.normal(size=(40, d, d))
    for energy, eps in (("sd", 2.0 ** -6.5), ("sg", 2.0 ** -13)):
        U, P = admm.polar_init(J, energy)
        det = np.linalg.det(J)
        ok = det > 0
        np.testing.assert_allclose(np.linalg.det(U), 1.0, atol=1e-12)
        np.testing.assert_allclose(np.transpose(U, (0, 2, 1)) @ U, np.broadcast_to(np.eye(d), U.shape), atol=1e-12)
        # unflipped: U P is the polar decomposition of J (unique), singular values >= eps
        sv = np.linalg.svd(J[ok], compute_uv=False)
        if np.all(sv > eps):
            np.testing.assert_allclose(U[ok] @ P[ok], J[ok], atol=1e-12)
        # flipped: P = eps I and U = polar factor with the last column negated
        np.testing.assert_allclose(P[~ok], np.broadcast_to(eps * np.eye(d), P[~ok].shape), atol=1e-15)
        R1, s, R2t = np.linalg.svd(J[~ok])
        O = R1 @ R2t
        O[:, :, -1] *= -1
        np.testing.assert_allclose(U[~ok], O, atol=1e-12)


def _sym_power(A, p):
    """A^p for a batch of symmetric positive definite matrices, via eigh."""
    lam, E = np.linalg.eigh(A)
    return np.einsum("mij,mj,mkj->mik", E, lam ** p, E)


def _random_orthogonal(rng, d, count, det_sign):
    Q, R = np.linalg.qr(rng.normal(size=(count, d, d)))
    Q = Q * np.sign(np.diagonal(R, axis1=1, axis2=2))[:, None, :]
    wrong = np.sign(np.linalg.det(Q)) != det_sign
    Q[wrong, :, 0] *= -1.0
    return Q


@pytest.mark.parametrize("d", [2, 3])
def test_polar_init_against_the_closed_form_polar_factor(d):
    """Eqs. initialpolardecomposition / polardecompositionapplied without an SVD:
    the orthogonal polar factor of an invertible J is J (J^T J)^{-1/2} and its
    symmetric factor (J^T J)^{1/2} (both from eigh of J^T J).  Unflipped: U is that
    factor (a rotation) and P has the eigenvalues of (J^T J)^{1/2} raised to eps.
    Flipped (det J < 0): the polar factor is a reflection, the best one for J
    (tr(O^T J) >= tr(Q^T J) for every reflection Q), and U is it with its last
    column negated, so det U = 1 and U diag(1, .., 1, -1) recovers it."""
    rng = np.random.default_rng(12)
    # well-conditioned draws plus some with one tiny singular value (below eps)
    J = rng.normal(size=(60, d, d))
    Qa = _random_orthogonal(rng, d, 20, 1.0)
    Qb = _random_orthogonal(rng, d, 20, 1.0)
    sv = np.abs(rng.normal(size=(20, d))) + 0.5
    sv[:, -1] = 1e-9
    J = np.concatenate([J, np.einsum("mij,mj,mkj->mik", Qa, sv, Qb)])
    J[-5:, :, 0] *= -1.0          # a few near-singular flipped ones too
    D = np.diag([1.0] * (d - 1) + [-1.0])
    JtJ = np.transpose(J, (0, 2, 1)) @ J
    lam, E = np.linalg.eigh(JtJ)
    det = np.linalg.det(J)
    # the closed form J (J^T J)^{-1/2} loses accuracy as J nears singularity, so
    # the polar factor is checked where the smallest singular value is above 1e-3
    good = lam[:, 0] > 1e-6
    O = np.full_like(J, np.nan)
    O[good] = J[good] @ _sym_power(JtJ[good], -0.5)
    pos, neg = det > 0, det < 0
    assert (pos & good).sum() > 10 and (neg & good).sum() > 10 and (pos & ~good).sum() > 5
    for energy, eps in (("sd", 2.0 ** -6.5), ("sg", 2.0 ** -13)):
        U, P = admm.polar_init(J, energy)
        # unflipped: U = J (J^T J)^{-1/2}, P = (J^T J)^{1/2} with eigenvalues raised to eps
        np.testing.assert_allclose(U[pos & good], O[pos & good], atol=1e-9)
        P_ref = np.einsum("mij,mj,mkj->mik", E, np.maximum(np.sqrt(np.maximum(lam, 0.0)), eps), E)
        np.testing.assert_allclose(P[pos], P_ref[pos], atol=1e-9)
        # flipped: O is a reflection, the best reflection for J, and U = O with its last column negated
        fl = neg & good
        np.testing.assert_allclose(np.linalg.det(O[fl]), -1.0, atol=1e-9)
        Qs = _random_orthogonal(rng, d, 4000, -1.0)
        for k in np.flatnonzero(fl):
            trials = np.einsum("qij,ij->q", Qs, J[k])
            assert np.all(trials <= np.einsum("ij,ij->", O[k], J[k]) + 1e-12)
        np.testing.assert_allclose(np.linalg.det(U[neg]), 1.0, atol=1e-12)
        np.testing.assert_allclose(U[fl] @ D, O[fl], atol=1e-9)
        np.testing.assert_allclose(P[neg], np.broadcast_to(eps * np.eye(d), P[neg].shape), atol=1e-15)


# --------------------------------------------------------------------------
# W step (eq. solvinginw) against a dense least-squares solve
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 1, 2])
def test_w_step_is_the_constrained_least_squares_minimizer(k):
    V, T = _small_meshes()[k]
    n = V.shape[0]
    d = T.shape[1] - 1
    g, w = admm.element_gradients(V, T)
    rng = np.random.default_rng(12)
    mu = w * rng.uniform(0.5, 3.0, size=len(w))
    pins = np.array([0, n - 1, n // 2])
    pin_pos = rng.normal(size=(3, d))
    ws = admm.WStep(g, T, mu, n, pins, pin_pos)
    Y = rng.normal(size=(T.shape[0], d, d))        # the target U P - Lambda
    W = ws.solve(admm.gradient_adjoint(g, T, mu[:, None, None] * Y, n))
    # dense: minimize sum_i mu_i |J_i(W) - Y_i|^2 over the free rows, columns independently
    free = np.setdiff1d(np.arange(n), pins)
    sq = np.sqrt(mu)[:, None]
    for c in range(d):
        cols = []
        for v in free:
            E = np.zeros((n, d))
            E[v, c] = 1.0
            cols.append((sq[:, :, None] * admm.jacobians(g, T, E)).ravel())
        A = np.stack(cols, 1)
        base = np.zeros((n, d))
        base[pins, c] = pin_pos[:, c]
        tgt = (sq[:, :, None] * (Y - admm.jacobians(g, T, base))).ravel()
        x = np.linalg.lstsq(A, tgt, rcond=None)[0]
        np.testing.assert_allclose(W[free, c], x, rtol=1e-9, atol=1e-10)
    np.testing.assert_array_equal(W[pins], pin_pos)


def test_w_step_without_pins_fixes_vertex_zero():
    V, T = _small_meshes()[0]
    g, w = admm.element_gradients(V, T)
    ws = admm.WStep(g, T, w, V.shape[0], np.array([], int), np.zeros((0, 2)))
    rng = np.random.default_rng(13)
    W = ws.solve(rng.normal(size=(V.shape[0], 2)))
    np.testing.assert_array_equal(W[0], [0.0, 0.0])


# --------------------------------------------------------------------------
# whole iterations
# --------------------------------------------------------------------------

@pytest.mark.parametrize("energy", ["sd", "sg", "sa"])
@pytest.mark.parametrize("k", [0, 1])
def test_rigid_motion_is_a_fixed_point(energy, k):
    """J in SO(d) gives q = 1 -> p = 1 for both energies: one iteration changes nothing,
    e_prim = 0, and the energy is sum w f(I) (zero distortion excess)."""
    V, T = _small_meshes()[k]
    d = V.shape[1]
    R = Rotation.from_rotvec([0.2, 0.5, -0.4]).as_matrix() if d == 3 else admm.rot2(np.array([0.8]), np.array([0.6]))[0]
    W0 = V @ R.T + 0.3
    pins = np.array([0, 3])
    o = admm.Oracle(V, T, pins, W0[pins], energy, rho=1.0)
    s0 = o.init(W0)
    s1, st = o.step(s0)
    np.testing.assert_allclose(s1.W, W0, atol=1e-12)
    np.testing.assert_allclose(s1.P, np.broadcast_to(np.eye(d), s1.P.shape), atol=1e-12)
    assert st.e_prim < 1e-11 and st.e_dual < 1e-11 and st.n_flipped == 0
    fI = {"sd": d, "sg": d / 2, "sa": 0.0}[energy]
    assert math.isclose(o.energy(s1.W), fI * o.w.sum(), rel_tol=1e-12, abs_tol=1e-20)


def _c1_small(rho=1.0):
    return wk.uv_disk(grid=16, seed=21, rho=rho)


def test_local_output_is_flip_free_and_kkt_holds():
    """Every P_i is SPD, det(U_i P_i) > 0 (Sec. 4, robustness), and after each iteration
    w grad f(P) = mu symm(U^T Lambda) holds (stationarity of the P step)."""
    wl = _c1_small()
    assert wl.meta["flipped0"] > 0
    o = admm.Oracle.from_workload(wl)
    checked = []

    def cb(k, s0, s1, st):
        ev = np.linalg.eigvalsh(s1.P)
        assert ev.min() > 0
        assert np.all(np.linalg.det(s1.U @ s1.P) > 0)
        lhs = o.w[:, None, None] * admm.grad_f(s1.P, wl.energy)
        rhs = o.mu[:, None, None] * admm.symm(np.transpose(s1.U, (0, 2, 1)) @ s1.Lam)
        assert np.abs(lhs - rhs).max() <= 1e-9 * max(1e-30, np.abs(lhs).max())
        checked.append(k)

    o.run(wl.W0, 30, stop_at_tol=False, callback=cb)
    assert len(checked) == 30


def test_convergence_unflips_and_meets_thresholds():
    """Fig. 3 / Sec. 6: from an initial map with flipped triangles the iteration removes the
    flips and drives e_prim and e_dual below the thresholds of eq. primaldualthresholds."""
    wl = wk.uv_disk(grid=24, seed=22, rho=3.0)
    assert wl.meta["flipped0"] > 0.01
    o = admm.Oracle.from_workload(wl)
    hist = []
    s, st = o.run(wl.W0, 400, callback=lambda k, a, b, t: hist.append(t))
    assert st.converged and st.n_flipped == 0
    assert st.k < 400
    assert hist[-1].e_prim < hist[0].e_prim * 1e-3
    assert math.isfinite(o.energy(s.W))


def test_energy_gradient_matches_finite_differences():
    V, T = _small_meshes()[1]
    o = admm.Oracle(V, T, np.array([0]), V[:1], "sd")
    rng = np.random.default_rng(14)
    W = V + 0.02 * rng.normal(size=V.shape)
    G = o.energy_gradient(W)
    h = 1e-6
    for _ in range(10):
        v, c = rng.integers(V.shape[0]), rng.integers(3)
        E = np.zeros_like(W)
        E[v, c] = h
        fd = (o.energy(W + E) - o.energy(W - E)) / (2 * h)
        assert abs(fd - G[v, c]) < 1e-6 * max(1.0, abs(G[v, c]))


def test_energy_is_infinite_when_flipped():
    V, T = _small_meshes()[0]
    o = admm.Oracle(V, T, np.array([0]), V[:1], "sg")
    W = V.copy()
    W[:, 0] *= -1
    assert o.energy(W) == math.inf


@pytest.mark.parametrize("k", [0, 1])
def test_local_steps_minimize_the_augmented_lagrangian(k):
    """U^k and P^k are the minimizers of Phi in U (eq. rawoptimizationinudecoupled, h = 0) and in P (eq. optimizinginp),
    found by brute force on the raw objective |J - U P + Lambda|^2, not through Q or S."""
    V, T = _small_meshes()[k]
    d = V.shape[1]
    rng = np.random.default_rng(15)
    W0 = V + 0.08 * rng.normal(size=V.shape)
    o = admm.Oracle(V, T, np.array([0, 1]), W0[:2], "sd", rho=2.0)
    s = o.init(W0)
    for _ in range(3):
        s, _ = o.step(s)
    W = o.w_step(s)
    s1 = o.local_steps(s, W)
    for i in range(3):
        J, Lam, P0, mu, w = s1.J[i], s.Lam[i], s.P[i], o.mu[i], o.w[i]
        phiU = lambda U: np.sum((J - U @ P0 + Lam) ** 2)
        if d == 3:
            Rs = Rotation.random(20000, random_state=16).as_matrix()
            x0 = Rotation.from_matrix(Rs[int(np.argmin([phiU(R) for R in Rs]))]).as_rotvec()
            r = so.minimize(lambda v: phiU(Rotation.from_rotvec(v).as_matrix()), x0, method="Nelder-Mead",
                            options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
            best = r.fun
        else:
            phis = np.linspace(0, 2 * math.pi, 400001)
            best = min(phiU(admm.rot2(np.array([math.cos(a)]), np.array([math.sin(a)]))[0]) for a in phis[::40])
            best = min(best, min(phiU(admm.rot2(np.cos(phis[j:j + 1]), np.sin(phis[j:j + 1]))[0])
                                 for j in range(0, len(phis), 997)))
        assert phiU(s1.U[i]) <= best + 1e-9 * max(1, best)
        U = s1.U[i]
        phiP = lambda x: w * admm.f_energy(_spd_from_params(x, d)[None], "sd")[0] + \
            0.5 * mu * np.sum((J - U @ _spd_from_params(x, d) + Lam) ** 2)
        r = so.minimize(phiP, rng.normal(scale=0.1, size=d * (d + 1) // 2), method="BFGS",
                        options=dict(gtol=1e-12, maxiter=20000))
        mineP = w * admm.f_energy(s1.P[i][None], "sd")[0] + 0.5 * mu * np.sum((J - U @ s1.P[i] + Lam) ** 2)
        assert mineP <= r.fun + 1e-12 * max(1, abs(r.fun))
        np.testing.assert_allclose(s1.P[i], _spd_from_params(r.x, d), atol=1e-4)
    # Lambda update and the primal error agree: e_prim = |Lambda^k - Lambda^{k-1}|
    st = o.stats(s, s1)
    assert math.isclose(st.e_prim, math.sqrt(np.sum((s1.Lam - s.Lam) ** 2)), rel_tol=1e-12)
