"""FP64 CPU oracle of the flip-free splitting scheme (Stein, Li & Solomon, 2021).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plainly written reference
that the CUDA path is checked against.  Only the test-suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the library never does.
It shares no code with the CUDA path: the only common module is the seeded
input generator, which holds none of the method's arithmetic.

Everything is IEEE double precision (Sec. 6: the paper computes in double).
Element data are batched numpy arrays; numpy/scipy primitives (SVD, symmetric
eigendecomposition, sparse LU) serve as single steps, and the steps follow the
paper's order (Algorithm 1 / Algorithm 2 without the rescaling branch).

Notation (Sec. 3.1 and its definition of the Jacobian): V source vertices (n, d_in), W target vertices
(n, d), T elements (m, d+1), w_i element area/volume, J = GW the per-element
Jacobians with column k equal to the gradient of target coordinate k
(Supplemental, "Computing the Jacobian map").  U_i in SO(d), P_i SPD, Lambda_i
the scaled multiplier, mu_i the penalties (eq. augmentedlagrangian).

Readings of points the paper leaves open (each one is also listed in the
design notes):
  * mu_i = rho * w_i, fixed (no rescaling); rho = 1 gives the paper's initial
    penalties mu_i = w_i (Sec. 6, rescaling paragraph).
  * h_i = 0 unless a proximal weight is passed (Sec. 6: disabled when many
    flipped elements are expected).
  * eps_m is the double-precision machine epsilon 2^-52 for every constant.
  * sqrt(d m) in the thresholds of eq. primaldualthresholds is taken literally.
  * 2D Procrustes tie (Q with q11+q22 = q21-q12 = 0): keep the previous U.
  * Flipped init: R1 R2^T gets its last column negated when its determinant is
    negative, and Sigma = eps I whenever det J0 <= 0.
  * General constraints A W = b (Sec. 4, W update): A is c x n and acts on every
    coordinate column alike, b is c x d (the paper's notation); constraints that
    mix coordinates are not covered.  Pinned vertices are rows of the identity.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

EPS_M = 2.0 ** -52
SQRT_EPS_M = 2.0 ** -26


# ----------------------------------------------------------------------------
# mesh operators (Supplemental, "Computing the Jacobian map"; Sec. 3.1, the Jacobian)
# ----------------------------------------------------------------------------

def element_frames(V: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Source edge vectors E_i = [v1-v0, ..., vd-v0] as rows, in the element frame.

    Volumes (d_in = d = 3) and planar triangles (d_in = d = 2) use the coordinate
    frame.  Surface triangles (d_in = 3, d = 2) use the intrinsic frame
    e1 = (v1-v0)/|v1-v0|, e2 = n x e1 with n the unit normal of (v1-v0) x (v2-v0).
    Returns (m, d, d) with row j the j-th edge vector.
    """
    d = T.shape[1] - 1
    E = V[T[:, 1:]] - V[T[:, :1]]              # (m, d, d_in)
    if V.shape[1] == d:
        return E
    assert d == 2 and V.shape[1] == 3
    e1 = E[:, 0] / np.linalg.norm(E[:, 0], axis=1, keepdims=True)
    nrm = np.cross(E[:, 0], E[:, 1])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    e2 = np.cross(nrm, e1)
    B = np.stack([e1, e2], axis=2)             # (m, 3, 2) columns e1, e2
    return np.einsum("mjk,mkl->mjl", E, B)


def element_gradients(V: np.ndarray, T: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Gradients of the P1 hat functions and element measures.

    For element i with edge matrix E_i (rows v_j - v_0, j = 1..d), the hat
    function of vertex j has a gradient g_j with g_j . (v_k - v_0) = delta_jk,
    i.e. g_j is column j of E_i^{-1}; g_0 = -sum_j g_j.  w_i = |det E_i| / d!.
    Returns g (m, d+1, d) and w (m,).
    """
    E = element_frames(V, T)
    d = E.shape[1]
    Einv = np.linalg.inv(E)                    # columns of E^{-1} are the g_j
    gj = np.transpose(Einv, (0, 2, 1))         # row j = g_{j+1}
    g0 = -gj.sum(axis=1, keepdims=True)
    g = np.concatenate([g0, gj], axis=1)
    w = np.abs(np.linalg.det(E)) / math.factorial(d)
    return g, w


def jacobians(g: np.ndarray, T: np.ndarray, W: np.ndarray) -> np.ndarray:
    """J_i = (G W)_i with J[a, k] = sum_j g_ij[a] W[T_ij, k] (column k = grad W_k)."""
    return np.einsum("mja,mjk->mak", g, W[T])


def gradient_adjoint(g: np.ndarray, T: np.ndarray, R: np.ndarray, n: int) -> np.ndarray:
    """G^T R for a matrix collection R: out[v, k] = sum_{(i,j): T_ij = v} g_ij . R_i[:, k]."""
    contrib = np.einsum("mja,mak->mjk", g, R)  # (m, d+1, d)
    out = np.zeros((n, R.shape[2]))
    np.add.at(out, T.ravel(), contrib.reshape(-1, R.shape[2]))
    return out


def assemble_L(g: np.ndarray, T: np.ndarray, mu: np.ndarray, n: int) -> sp.csr_matrix:
    """L = sum_i mu_i G_i^T G_i (eq. solvinginw): L[u, v] += mu_i g_iu . g_iv."""
    k = T.shape[1]
    loc = mu[:, None, None] * np.einsum("mja,mla->mjl", g, g)
    rows = np.repeat(T, k, axis=1).ravel()
    cols = np.tile(T, (1, k)).ravel()
    return sp.csr_matrix((loc.ravel(), (rows, cols)), shape=(n, n))


# ----------------------------------------------------------------------------
# defining functions and gradients (eqs. symmetricgradientdefiningfunction/symmetricgradientdefininggrad, eqs. symmetricdirichletdefiningfunction/symmetricdirichletdefininggrad)
# ----------------------------------------------------------------------------

def rotation_part(X: np.ndarray) -> np.ndarray:
    """R(X): the rotation of the polar decomposition X = R S (det X > 0), U V^T of the SVD."""
    U, _, Vt = np.linalg.svd(X)
    return U @ Vt


def f_energy(X: np.ndarray, energy: str) -> np.ndarray:
    """f_SD(X) = (|X|^2 + |X^-1|^2)/2 ;  f_SG(X) = |X|^2/2 - log det X ;
    f_SA(X) = (|X - R|^2 + |X^-1 - R^-1|^2)/2 with R the rotation of X (the
    symmetric ARAP energy, one more rotation-invariant choice of the defining
    function, Sec. 3: other energies plug into the same scheme)."""
    fro2 = np.einsum("mij,mij->m", X, X)
    if energy == "sd":
        Xi = np.linalg.inv(X)
        return 0.5 * (fro2 + np.einsum("mij,mij->m", Xi, Xi))
    if energy == "sa":
        R = rotation_part(X)
        D1 = X - R
        D2 = np.linalg.inv(X) - np.transpose(R, (0, 2, 1))
        return 0.5 * (np.einsum("mij,mij->m", D1, D1) + np.einsum("mij,mij->m", D2, D2))
    return 0.5 * fro2 - np.log(np.linalg.det(X))


def grad_f(X: np.ndarray, energy: str) -> np.ndarray:
    """grad f_SD = X - X^-T X^-1 X^-T ;  grad f_SG = X - X^-T ;
    grad f_SA = U diag(phi'(s)) V^T for X = U diag(s) V^T, phi'(s) = s - 1 - s^-3 + s^-2
    (f_SA = sum phi(s_k), phi(s) = ((s - 1)^2 + (1/s - 1)^2)/2)."""
    if energy == "sa":
        U, sv, Vt = np.linalg.svd(X)
        dphi = sv - 1.0 - sv ** -3 + sv ** -2
        return np.einsum("mij,mj,mjk->mik", U, dphi, Vt)
    XiT = np.transpose(np.linalg.inv(X), (0, 2, 1))
    if energy == "sd":
        Xi = np.linalg.inv(X)
        return X - XiT @ Xi @ XiT
    return X - XiT


def energy(g, T, W, w, energy_name: str) -> float:
    """E(W) = sum_i w_i f((GW)_i) + chi_+(det (GW)_i)  (eq. genericdeformationenergy)."""
    J = jacobians(g, T, W)
    if np.any(np.linalg.det(J) <= 0.0):
        return math.inf
    return float(np.sum(w * f_energy(J, energy_name)))


def energy_gradient(g, T, W, w, energy_name: str) -> np.ndarray:
    """dE/dW = G^T (w_i grad f(J_i)), defined where every det J_i > 0."""
    J = jacobians(g, T, W)
    if np.any(np.linalg.det(J) <= 0.0):
        raise ValueError("energy gradient undefined: flipped element")
    return gradient_adjoint(g, T, w[:, None, None] * grad_f(J, energy_name), W.shape[0])


# ----------------------------------------------------------------------------
# local steps (Sec. 4 and Supplemental)
# ----------------------------------------------------------------------------

def rot2(c: np.ndarray, s: np.ndarray) -> np.ndarray:
    return np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)


def procrustes(Q: np.ndarray, U_prev: np.ndarray) -> np.ndarray:
    """argmin_{U in SO(d)} |U - Q|^2 (eq. optimizationinudecoupled).

    d = 2: U(phi) maximizes U(phi).Q = cos(phi)(q11+q22) + sin(phi)(q21-q12),
    so (cos, sin) is that vector normalized (Supplemental, d = 2); a zero vector
    means every rotation is optimal and U_prev is kept.
    d = 3: SVD Q = R1 S R2^T and U = R1 diag(1, 1, det(R1 R2^T)) R2^T.
    """
    d = Q.shape[1]
    if d == 2:
        a = Q[:, 0, 0] + Q[:, 1, 1]
        b = Q[:, 1, 0] - Q[:, 0, 1]
        r = np.hypot(a, b)
        U = U_prev.copy()
        ok = r > 0
        U[ok] = rot2(a[ok] / r[ok], b[ok] / r[ok])
        return U
    R1, _, R2t = np.linalg.svd(Q)
    sgn = np.sign(np.linalg.det(R1 @ R2t))
    sgn[sgn == 0] = 1.0
    D = np.zeros_like(Q)
    D[:, 0, 0] = 1.0
    D[:, 1, 1] = 1.0
    D[:, 2, 2] = sgn
    return R1 @ D @ R2t


def root_sg(q: np.ndarray, w: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Positive root of (w+mu) p^2 - mu q p - w = 0 (eq. peqfsgpluggedin per eigenvalue, eq. solvesgwithquadraticformula).

    For q >= 0 the quadratic formula as printed; for q < 0 the algebraically equal
    form 2w / (sqrt(disc) - mu q), which avoids cancelling two large terms.
    """
    disc = np.sqrt(mu * mu * q * q + 4.0 * w * (w + mu))
    plus = (mu * q + disc) / (2.0 * (w + mu))
    minus = 2.0 * w / (disc - mu * q)
    return np.where(q >= 0.0, plus, minus)


def root_sd(q: np.ndarray, w: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Unique positive root of (w+mu) p^4 - mu q p^3 - w = 0 (eq. peqfsdpluggedin per eigenvalue).

    With a = mu q/(w+mu) and c = w/(w+mu) the root lies in
    (0, max(a, 0) + c^{1/4}]: the quartic is -c < 0 at 0, and at
    p = max(a,0) + c^{1/4} it is p^3 (p - a) - c >= c^{3/4} c^{1/4} - c = 0.
    Bisection to adjacent doubles, then one Newton step from the midpoint.
    """
    a = mu * q / (w + mu)
    c = w / (w + mu)
    lo = np.zeros_like(q)
    hi = np.maximum(a, 0.0) + c ** 0.25

    def g(p):
        return p ** 3 * (p - a) - c

    for _ in range(200):
        mid = 0.5 * (lo + hi)
        neg = g(mid) < 0.0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
        if np.all(np.nextafter(lo, np.inf) >= hi):
            break
    p = 0.5 * (lo + hi)
    dg = p * p * (4.0 * p - 3.0 * a)
    step = np.where(dg > 0, g(p) / np.where(dg > 0, dg, 1.0), 0.0)
    pn = p - step
    return np.where((pn >= lo) & (pn <= hi), pn, p)


def root_sa(q: np.ndarray, w: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Unique positive root of (w+mu) p^4 - (w + mu q) p^3 + w p - w = 0: the
    stationarity condition w phi'(p) + mu (p - q) = 0 of the symmetric ARAP
    scalar prox, multiplied by p^3.

    With a = (w + mu q)/(w+mu) and c = w/(w+mu) it reads g(p) = p^3 (p - a) +
    c (p - 1) = 0; g(0) = -c < 0 and g(max(1, a)) >= 0, so the root lies in
    (0, max(1, a)] (the objective w phi(p) + mu/2 (p - q)^2 is strictly convex on
    p > 0, so there is one).  Bisection to adjacent doubles, then one Newton step.
    """
    a = (w + mu * q) / (w + mu)
    c = w / (w + mu)
    lo = np.zeros_like(q)
    hi = np.maximum(a, 1.0)

    def g(p):
        return p ** 3 * (p - a) + c * (p - 1.0)

    for _ in range(200):
        mid = 0.5 * (lo + hi)
        neg = g(mid) < 0.0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
        if np.all(np.nextafter(lo, np.inf) >= hi):
            break
    p = 0.5 * (lo + hi)
    dg = p * p * (4.0 * p - 3.0 * a) + c
    step = np.where(dg > 0, g(p) / np.where(dg > 0, dg, 1.0), 0.0)
    pn = p - step
    return np.where((pn >= lo) & (pn <= hi), pn, p)


def p_step(S: np.ndarray, w: np.ndarray, mu: np.ndarray, energy_name: str) -> np.ndarray:
    """argmin_{P SPD} w f(P) + mu/2 |P - S|^2 for symmetric S (eqs. optimizinginp/rootfindinginp, Supplemental).

    S = E diag(q) E^T; each eigenvalue is mapped to the positive root of the
    scalar version of eq. peqfsgpluggedin/(S.4); if det P or tr P falls below sqrt(eps_m)
    the eigenvalues are raised to at least sqrt(eps_m).
    """
    q, E = np.linalg.eigh(S)
    ww = w[:, None] * np.ones_like(q)
    mm = mu[:, None] * np.ones_like(q)
    roots = {"sg": root_sg, "sd": root_sd, "sa": root_sa}
    p = roots[energy_name](q, ww, mm)
    small = (np.prod(p, axis=1) < SQRT_EPS_M) | (np.sum(p, axis=1) < SQRT_EPS_M)
    p[small] = np.maximum(p[small], SQRT_EPS_M)
    return np.einsum("mij,mj,mkj->mik", E, p, E)


def symm(X: np.ndarray) -> np.ndarray:
    return 0.5 * (X + np.transpose(X, (0, 2, 1)))


def polar_init(J0: np.ndarray, energy_name: str) -> tuple[np.ndarray, np.ndarray]:
    """U0, P0 from the polar decomposition of GW0 (eqs. initialpolardecomposition/polardecompositionapplied).

    J0 = R1 S R2^T, U0 = R1 R2^T, P0 = R2 S R2^T; singular values below eps are
    raised to eps, eps = eps_m^{1/4} (SG) or eps_m^{1/8} (SD, and SA, which grows
    like SD as a singular value goes to 0).  A flipped J0
    (det <= 0) gets S = eps I and, when R1 R2^T is a reflection, its last column
    negated.
    """
    eps = EPS_M ** 0.25 if energy_name == "sg" else EPS_M ** 0.125
    R1, s, R2t = np.linalg.svd(J0)
    O = R1 @ R2t
    flipped = np.linalg.det(J0) <= 0.0
    refl = np.linalg.det(O) < 0.0
    O[refl, :, -1] *= -1.0
    s = np.maximum(s, eps)
    s[flipped] = eps
    R2 = np.transpose(R2t, (0, 2, 1))
    P0 = np.einsum("mij,mj,mkj->mik", R2, s, R2)
    return O, P0


# ----------------------------------------------------------------------------
# global step (eq. solvinginw with constraints A W = b as pinned vertices)
# ----------------------------------------------------------------------------

class WStep:
    """Exact minimizer of Phi over W with pinned vertices (eq. solvinginw).

    L = sum mu_i G_i^T G_i is split into free (F) and pinned (C) blocks;
    L_FF W_F = (G^T r)_F - L_FC b.  L_FF is factored once (sparse LU), as the
    paper decomposes L once and back-substitutes every iteration (Sec. 4).
    With no pins, vertex 0 is fixed at the origin (Sec. 4, W update).
    """

    def __init__(self, g, T, mu, n, pins, pin_pos):
        if len(pins) == 0:
            pins = np.array([0], dtype=np.int64)
            pin_pos = np.zeros((1, g.shape[2]))
        self.n = n
        self.pins = np.asarray(pins, dtype=np.int64)
        self.pin_pos = np.asarray(pin_pos, dtype=np.float64)
        mask = np.ones(n, bool)
        mask[self.pins] = False
        self.free = np.nonzero(mask)[0]
        L = assemble_L(g, T, mu, n)
        self.L = L
        self.L_FF = L[self.free][:, self.free].tocsc()
        self.L_FC = L[self.free][:, self.pins]
        self.lu = sla.splu(self.L_FF, permc_spec="MMD_AT_PLUS_A")

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        W = np.zeros((self.n, rhs.shape[1]))
        W[self.pins] = self.pin_pos
        b = rhs[self.free] - self.L_FC @ self.pin_pos
        W[self.free] = self.lu.solve(np.ascontiguousarray(b))
        return W


class WStepKKT:
    """Exact minimizer of Phi over W subject to general linear constraints
    A W = b (Sec. 4, W update: any feasible A W = b; A is c x n and acts on every
    coordinate column alike, b is c x d).  The KKT system

        [ L  A^T ] [ W   ]   [ G^T r ]
        [ A  0   ] [ nu  ] = [ b     ]

    is indefinite; it is factored once by sparse LU (the paper's UMFPACK role)
    and back-substituted every iteration.  Pinned vertices are rows of the
    identity in A.  Raises ValueError when the system is singular (the
    constraints do not fix the translations that G annihilates).
    """

    def __init__(self, g, T, mu, n, A, b):
        A = sp.csr_matrix(A, dtype=np.float64)
        if A.shape[1] != n:
            raise ValueError("A must have n columns")
        self.n = n
        self.A = A
        self.b = np.asarray(b, dtype=np.float64)
        L = assemble_L(g, T, mu, n)
        self.L = L
        # L annihilates the constant vectors (a connected mesh), so the system is
        # regular only if some constraint row has a nonzero sum, and only if the
        # rows are independent (checked on the pivots of the factorization)
        if np.abs(A @ np.ones(n)).max() <= 1e-12 * max(1.0, abs(A).max()):
            raise ValueError("singular constrained W step: the constraints fix no translation")
        K = sp.bmat([[L, A.T], [A, None]], format="csc")
        try:
            self.lu = sla.splu(K, permc_spec="MMD_AT_PLUS_A")
        except RuntimeError as e:   # exactly singular
            raise ValueError(f"singular constrained W step: dependent constraints ({e})") from e
        piv = np.abs(self.lu.U.diagonal())
        if not np.all(np.isfinite(piv)) or piv.min() <= 1e-13 * piv.max():
            raise ValueError("singular constrained W step: dependent constraints")

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        top = np.vstack([rhs, self.b])
        sol = self.lu.solve(np.ascontiguousarray(top))
        return sol[: self.n]


def pin_rows(pins, n: int) -> sp.csr_matrix:
    """The constraint rows of pinned vertices: one row of the identity per pin."""
    pins = np.asarray(pins, dtype=np.int64)
    return sp.csr_matrix((np.ones(len(pins)), (np.arange(len(pins)), pins)), shape=(len(pins), n))


# ----------------------------------------------------------------------------
# the loop (Algorithm 1; Algorithm 2 without rescaling)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class State:
    W: np.ndarray
    U: np.ndarray
    P: np.ndarray
    Lam: np.ndarray
    J: np.ndarray          # (G W^{(k)})_i, kept for the dual error of the next step


@dataclasses.dataclass
class Stats:
    k: int
    e_prim: float
    e_dual: float
    thr_prim: float
    thr_dual: float
    n_flipped: int
    energy_P: float
    converged: bool


class Oracle:
    """The FP64 reference solver for one mesh, one energy, fixed penalties."""

    def __init__(self, V, T, pins, pin_pos, energy_name: str, rho: float = 1.0,
                 eps_abs: float = 1e-6, eps_rel: float = 1e-5, h=None, local_variant: str = "paper",
                 constraints=None):
        self.V = np.asarray(V, np.float64)
        self.T = np.asarray(T, np.int64)
        self.energy_name = energy_name
        self.g, self.w = element_gradients(self.V, self.T)
        if np.any(self.w <= 0):
            raise ValueError("degenerate source element")
        self.n = self.V.shape[0]
        self.m, self.d = self.T.shape[0], self.T.shape[1] - 1
        self.mu = rho * self.w
        self.h = np.zeros(self.m) if h is None else np.broadcast_to(h, (self.m,)).astype(float)
        self.eps_abs, self.eps_rel = eps_abs, eps_rel
        if local_variant not in ("paper", "joint"):
            raise ValueError("local_variant must be 'paper' or 'joint'")
        self.local_variant = local_variant
        if constraints is None:
            self.wstep = WStep(self.g, self.T, self.mu, self.n, np.asarray(pins), np.asarray(pin_pos))
        else:
            # general A W = b (the pins, if any, become rows of the identity in A)
            A, b = constraints
            A = sp.csr_matrix(A, dtype=np.float64)
            b = np.asarray(b, dtype=np.float64)
            if len(pins):
                A = sp.vstack([pin_rows(pins, self.n), A]).tocsr()
                b = np.vstack([np.asarray(pin_pos, np.float64), b])
            self.wstep = WStepKKT(self.g, self.T, self.mu, self.n, A, b)

    @classmethod
    def from_workload(cls, wl, **kw):
        kw.setdefault("eps_abs", wl.eps_abs)
        kw.setdefault("eps_rel", wl.eps_rel)
        return cls(wl.V, wl.T, wl.pins, wl.pin_pos, wl.energy, wl.rho, **kw)

    def init(self, W0) -> State:
        """U0, P0 by polar decomposition, Lambda0 = 0 (Algorithm 2, eqs. initialpolardecomposition/polardecompositionapplied)."""
        W0 = np.asarray(W0, np.float64)
        J0 = jacobians(self.g, self.T, W0)
        U0, P0 = polar_init(J0, self.energy_name)
        return State(W0.copy(), U0, P0, np.zeros_like(J0), J0)

    def w_step(self, s: State) -> np.ndarray:
        r = self.mu[:, None, None] * (s.U @ s.P - s.Lam)
        return self.wstep.solve(gradient_adjoint(self.g, self.T, r, self.n))

    def local_steps(self, s: State, W: np.ndarray) -> State:
        """U, P and Lambda updates for a given W^{(k)} (Sec. 4).

        local_variant "paper": the U step uses P^{k-1} (Algorithm 1).
        local_variant "joint" (not the paper's scheme): (U, P) minimize
        w f(P) + mu/2 |U P - A|^2 together.  For a rotation-invariant f the
        minimizer is U = the rotation nearest to A itself and P = the prox of
        symm(U^T A) (von Neumann's trace inequality: |U P - A|^2 is smallest when
        P shares A's right singular vectors, and then the P problem separates per
        signed singular value), so only Q changes; h is not used."""
        J = jacobians(self.g, self.T, W)
        A = J + s.Lam
        if self.local_variant == "joint":
            Q = A
        else:
            Q = A @ s.P + (self.h / self.mu)[:, None, None] * s.U
        U = procrustes(Q, s.U)
        S = symm(np.transpose(U, (0, 2, 1)) @ A)
        P = p_step(S, self.w, self.mu, self.energy_name)
        Lam = s.Lam + J - U @ P
        return State(W, U, P, Lam, J)

    def step(self, s: State) -> tuple[State, Stats]:
        W = self.w_step(s)
        s1 = self.local_steps(s, W)
        return s1, self.stats(s, s1)

    def stats(self, s0: State, s1: State, k: int = 0) -> Stats:
        """Primal/dual errors and thresholds (eqs. primaldualerror/primaldualthresholds), flips, sum w f(P)."""
        R = s1.J - s1.U @ s1.P
        e_prim = math.sqrt(np.sum(R * R))
        D = s1.J - s0.J
        e_dual = math.sqrt(np.sum((self.mu ** 2)[:, None, None] * D * D))
        base = self.eps_abs * math.sqrt(self.d * self.m)
        thr_p = base + self.eps_rel * max(math.sqrt(np.sum(s1.J * s1.J)),
                                          math.sqrt(np.sum(s1.P * s1.P)))
        GtL = gradient_adjoint(self.g, self.T, s1.Lam, self.n)
        thr_d = base + self.eps_rel * math.sqrt(np.sum(GtL * GtL))
        n_flip = int(np.sum(np.linalg.det(s1.J) <= 0.0))
        eP = float(np.sum(self.w * f_energy(s1.P, self.energy_name)))
        conv = e_prim < thr_p and e_dual < thr_d and n_flip == 0
        return Stats(k, e_prim, e_dual, thr_p, thr_d, n_flip, eP, conv)

    def condition_proxies(self, s0: State, s1: State, mu0=None, mu1=None) -> tuple[float, float]:
        """The two quantities the paper plots beside the errors as evidence for the
        conditions of its convergence analysis (Fig. 3; Sec. 5, Conditions 1 and 2):

          * max_i |grad f(P_i^{k+1})|, a proxy for the gradient bound B_i of
            Condition 1;
          * max_i of |D_i| / |(D_i + U_i^{k+1} M_i^{k+1 T} U_i^{k+1}
            - U_i^k M_i^{k T} U_i^k) / 2| with D_i = M_i^{k+1} - M_i^k, a proxy for
            gamma^{1/2} of Condition 2 (the smallest gamma that the step satisfies),
            where M_i = mu_i Lambda_i is the multiplier with this module's scaled
            Lambda multiplied back by the penalty, so that values compare across
            rescalings (mu0, mu1: the penalties of s0 and s1, default the current
            ones).  An element whose denominator vanishes with D_i != 0 makes the
            ratio infinite; elements with D_i = 0 are skipped.
        """
        mu0 = self.mu if mu0 is None else np.asarray(mu0, np.float64)
        mu1 = self.mu if mu1 is None else np.asarray(mu1, np.float64)
        G = grad_f(s1.P, self.energy_name)
        g = float(np.sqrt(np.sum(G * G, axis=(1, 2))).max())
        M0 = mu0[:, None, None] * s0.Lam
        M1 = mu1[:, None, None] * s1.Lam
        D = M1 - M0
        tr = lambda X: np.transpose(X, (0, 2, 1))
        S = 0.5 * (D + s1.U @ tr(M1) @ s1.U - s0.U @ tr(M0) @ s0.U)
        num = np.sqrt(np.sum(D * D, axis=(1, 2)))
        den = np.sqrt(np.sum(S * S, axis=(1, 2)))
        moved = num > 0.0
        if not moved.any():
            return g, 0.0
        if np.any(den[moved] == 0.0):
            return g, math.inf
        return g, float((num[moved] / den[moved]).max())

    def run(self, W0, max_iter: int, stop_at_tol: bool = True, callback=None):
        s = self.init(W0)
        st = None
        for k in range(1, max_iter + 1):
            s1, st = self.step(s)
            st.k = k
            if callback is not None:
                callback(k, s, s1, st)
            s = s1
            if stop_at_tol and st.converged:
                break
        return s, st

    def energy(self, W) -> float:
        return energy(self.g, self.T, np.asarray(W, np.float64), self.w, self.energy_name)

    def energy_gradient(self, W) -> np.ndarray:
        return energy_gradient(self.g, self.T, np.asarray(W, np.float64), self.w, self.energy_name)
