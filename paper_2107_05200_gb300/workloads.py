"""Seeded synthetic workloads (meshes, pins, initial maps) for the flip-free ADMM.

This module only builds inputs: source meshes V/T, pinned vertices with their
target positions, and the initial map W0.  It holds none of the splitting
method's arithmetic (no Jacobians, no local or global steps), so that both the
CUDA path and the FP64 oracle can be fed from it without sharing method code.

The paper's meshes and datasets (Table 2, Sec. 7) are not available, so these
workloads stand in for them.  Their shapes follow the paper's problem setup
(Sec. 3.1: triangle meshes mapped to the plane, tetrahedral meshes mapped to
R^3) and the initializers it uses (Sec. 6: Tutte embeddings; App. A, Tutte's energy).

Conventions (Sec. 3.1): V is (n, d_in) float64, T is (m, d+1) int32 with
positively oriented elements, W is (n, d_out) float64 row-major, pins are int32
vertex indices with target positions pin_pos (n_pin, d_out).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SYM_DIRICHLET = "sd"
SYM_GRADIENT = "sg"
SYM_ARAP = "sa"


@dataclasses.dataclass
class Workload:
    name: str
    V: np.ndarray          # (n, d_in) float64 source vertices
    T: np.ndarray          # (m, d+1) int32 elements
    pins: np.ndarray       # (n_pin,) int32 constrained vertices
    pin_pos: np.ndarray    # (n_pin, d_out) float64 constraint values b
    W0: np.ndarray         # (n, d_out) float64 initial map
    energy: str            # "sd", "sg" or "sa"
    rho: float = 1.0       # penalty scale, mu_i = rho * w_i
    eps_abs: float = 1e-6
    eps_rel: float = 1e-5
    max_iter: int = 500
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.V.shape[0]

    @property
    def m(self) -> int:
        return self.T.shape[0]

    @property
    def d(self) -> int:
        return self.T.shape[1] - 1

    @property
    def d_in(self) -> int:
        return self.V.shape[1]

    @property
    def d_out(self) -> int:
        return self.W0.shape[1]


# ----------------------------------------------------------------------------
# mesh builders
# ----------------------------------------------------------------------------

def grid_triangles(nx: int, ny: int, no_ears: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Regular triangulation of [0,1]^2 with nx*ny vertices, counter-clockwise.

    Every cell is split along its (0,0)-(1,1) diagonal.  With no_ears, the two
    corner cells whose split would give a triangle with all three vertices on
    the boundary use the other diagonal instead.
    """
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    V = np.stack([i.ravel() / (nx - 1), j.ravel() / (ny - 1)], axis=1).astype(np.float64)
    vid = (i * ny + j)
    v00 = vid[:-1, :-1].ravel()
    v10 = vid[1:, :-1].ravel()
    v11 = vid[1:, 1:].ravel()
    v01 = vid[:-1, 1:].ravel()
    T = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    if no_ears:
        ncell = (nx - 1) * (ny - 1)
        for ci, cj in ((nx - 2, 0), (0, ny - 2)):
            c = ci * (ny - 1) + cj
            a, b, cc, dd = v00[c], v10[c], v11[c], v01[c]
            T[c] = (a, b, dd)
            T[ncell + c] = (b, cc, dd)
    return V, T.astype(np.int32)


def _kuhn_cell_tets() -> list[tuple[int, int, int, int]]:
    """Six tetrahedra of the unit cell sharing the v000-v111 diagonal.

    Corners are numbered c = x + 2y + 4z.  Each permutation of the axes gives the
    monotone path v000 -> v000+e_a -> v000+e_a+e_b -> v111.  Odd permutations are
    reoriented by swapping the two middle vertices so every tet is positive.
    """
    tets = []
    perms = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]
    for k, p in enumerate(perms):
        a = 1 << p[0]
        b = a | (1 << p[1])
        t = (0, a, b, 7)
        if k >= 3:
            t = (0, b, a, 7)
        tets.append(t)
    return tets


def cube_tets(cells: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit cube split into cells^3 cubes, 6 Kuhn tetrahedra per cube."""
    k1 = cells + 1
    i, j, l = np.meshgrid(np.arange(k1), np.arange(k1), np.arange(k1), indexing="ij")
    V = np.stack([i.ravel(), j.ravel(), l.ravel()], 1).astype(np.float64) / cells
    vid = (i * k1 + j) * k1 + l
    corners = []
    for c in range(8):
        dx, dy, dz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        corners.append(vid[dx:cells + dx, dy:cells + dy, dz:cells + dz].ravel())
    tets = [np.stack([corners[a], corners[b], corners[c], corners[e]], 1)
            for (a, b, c, e) in _kuhn_cell_tets()]
    # element order: cell-major, so neighbouring elements share vertices
    T = np.stack(tets, 1).reshape(-1, 4)
    return V, T.astype(np.int32)


def _signed_measure(X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Signed area (2D) or signed volume (3D) of each element, from coordinates."""
    E = X[T[:, 1:]] - X[T[:, :1]]
    if T.shape[1] == 3:
        return 0.5 * (E[:, 0, 0] * E[:, 1, 1] - E[:, 0, 1] * E[:, 1, 0])
    return np.einsum("ij,ij->i", E[:, 0], np.cross(E[:, 1], E[:, 2])) / 6.0


def flipped_fraction(W: np.ndarray, T: np.ndarray) -> float:
    """Fraction of elements whose target orientation is non-positive."""
    return float(np.mean(_signed_measure(W, T) <= 0.0))


def _grid_boundary_cycle(nx: int, ny: int) -> np.ndarray:
    """Boundary vertex ids of an nx*ny grid in counter-clockwise cyclic order."""
    vid = np.arange(nx * ny).reshape(nx, ny)
    bottom = vid[:, 0]
    right = vid[-1, 1:]
    top = vid[-2::-1, -1]
    left = vid[0, -2:0:-1]
    return np.concatenate([bottom, right, top, left])


def _edges(T: np.ndarray) -> np.ndarray:
    k = T.shape[1]
    e = np.concatenate([T[:, [a, b]] for a in range(k) for b in range(a + 1, k)], 0)
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def tutte_embedding(V: np.ndarray, T: np.ndarray, boundary: np.ndarray,
                    boundary_pos: np.ndarray) -> np.ndarray:
    """Minimizer of the Tutte energy with fixed boundary (App. A, Tutte's energy).

    Edge weights are 1/|V_i - V_j|; interior vertices solve the weighted
    graph-Laplacian system.  Input construction only.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    n = V.shape[0]
    e = _edges(T)
    wgt = 1.0 / np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1)
    r = np.concatenate([e[:, 0], e[:, 1], e[:, 0], e[:, 1]])
    c = np.concatenate([e[:, 1], e[:, 0], e[:, 0], e[:, 1]])
    v = np.concatenate([-wgt, -wgt, wgt, wgt])
    Lt = sp.csr_matrix((v, (r, c)), shape=(n, n))
    is_b = np.zeros(n, bool)
    is_b[boundary] = True
    inner = np.nonzero(~is_b)[0]
    W = np.zeros((n, boundary_pos.shape[1]))
    W[boundary] = boundary_pos
    A = Lt[inner][:, inner].tocsc()
    rhs = -Lt[inner][:, boundary] @ boundary_pos
    W[inner] = np.column_stack([sla.spsolve(A, rhs[:, k]) for k in range(rhs.shape[1])])
    return W


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

def _noise_scale_for_flips(base: np.ndarray, xi: np.ndarray, T: np.ndarray,
                           target: float, hi: float, margin: float = 1e-6) -> float:
    """Noise scale s such that base + s*xi has the target fraction of flipped
    elements and no element sits at the flip threshold.

    Bisection finds the smallest s, to rounding, at which the flipped fraction
    reaches the target.  At that s one element's signed measure is zero up to
    rounding, so whether it counts as flipped would be decided by the order in
    which each program forms its determinant.  The scale is therefore moved past
    the crossing by relative steps of 1e-3 until every element's signed measure
    is at least `margin` times its measure in `base` away from zero.
    """
    lo = 0.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if flipped_fraction(base + mid * xi, T) < target:
            lo = mid
        else:
            hi = mid
    ref = np.abs(_signed_measure(base, T))
    for k in range(1, 500):
        s = hi * (1.0 + 1e-3 * k)
        if np.all(np.abs(_signed_measure(base + s * xi, T)) >= margin * ref):
            return s
    raise RuntimeError("no noise scale near the target keeps every element off the flip threshold")


def uv_disk(grid: int = 48, seed: int = 1, target_flip: float | None = 0.03,
            sigma: float = 0.05, jitter: float = 0.2,
            energy: str = SYM_DIRICHLET, rho: float = 1.0, max_iter: int = 500,
            tol: float = 1e-6) -> Workload:
    """2D plain method: jittered grid on [0,1]^2, boundary pinned to the unit circle.

    grid x grid vertices; interior vertices jittered uniformly by +-jitter cells.
    Boundary vertices keep their cyclic order and are placed on the unit circle by
    source arc length.  The two corner cells use the other diagonal so that no
    triangle has all three vertices pinned (such a triangle has a fixed Jacobian
    and its primal error can only shrink as its multiplier grows without bound).
    W0 = Tutte embedding plus Gaussian noise on the interior
    vertices.  With target_flip set, the noise scale is found by bisection on a
    fixed draw so that this fraction of triangles starts flipped; with
    target_flip=None the noise is N(0, sigma^2) in target units.
    """
    rng = np.random.default_rng(seed)
    V, T = grid_triangles(grid, grid, no_ears=True)
    h = 1.0 / (grid - 1)
    bnd = _grid_boundary_cycle(grid, grid)
    inner = np.ones(V.shape[0], bool)
    inner[bnd] = False
    V[inner] += rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 2))
    seg = np.linalg.norm(np.diff(V[np.r_[bnd, bnd[:1]]], axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)[:-1]]) / seg.sum()
    circ = np.stack([np.cos(2 * math.pi * s), np.sin(2 * math.pi * s)], 1)
    Wt = tutte_embedding(V, T, bnd, circ)
    xi = np.zeros_like(Wt)
    xi[inner] = rng.standard_normal(size=(inner.sum(), 2))
    if target_flip is not None:
        sigma = _noise_scale_for_flips(Wt, xi, T, target_flip, hi=1.0)
    W0 = Wt + sigma * xi
    wl = Workload(f"uv_disk_{grid}", V, T, bnd.astype(np.int32), circ, W0, energy, rho,
                  eps_abs=tol, eps_rel=10 * tol, max_iter=max_iter)
    wl.meta = dict(sigma=sigma, flipped0=flipped_fraction(W0, T),
                   tutte_flipped=flipped_fraction(Wt, T))
    return wl


def uv_heightfield(grid: int = 512, seed: int = 2, energy: str = SYM_GRADIENT,
                   target_flip: float = 0.05, rho: float = 10.0, max_iter: int = 2000,
                   tol: float = 1e-5) -> Workload:
    """2D UV-scale loop: grid^2 vertices on z = 0.3 sin(3x) cos(2y), flattened.

    Penalties mu_i = rho w_i with rho = 10: with rho = 1 or 3 (far below the
    penalty bound of the paper's convergence analysis, about 25 w_i for this
    energy at the rest state) the iteration oscillates without converging.
    Source V is the 3D surface (intrinsic 2x2 Jacobians).  Two pinned vertices,
    (0,0) and (grid-1,0), at their projected positions.  W0 = projection (x, y) plus
    Gaussian noise whose scale is found by bisection so that target_flip of the
    triangles start flipped (fixed noise draw, so the result is deterministic).
    """
    rng = np.random.default_rng(seed)
    P2, T = grid_triangles(grid, grid)
    z = 0.3 * np.sin(3 * P2[:, 0]) * np.cos(2 * P2[:, 1])
    V = np.column_stack([P2, z])
    pins = np.array([0, (grid - 1) * grid], dtype=np.int32)
    xi = rng.standard_normal(size=P2.shape)
    sigma = _noise_scale_for_flips(P2, xi, T, target_flip, hi=4.0 / (grid - 1))
    W0 = P2 + sigma * xi
    W0[pins] = P2[pins]
    wl = Workload(f"uv_heightfield_{grid}", V, T, pins, P2[pins].copy(), W0, energy, rho,
                  eps_abs=tol, eps_rel=10 * tol, max_iter=max_iter)
    wl.meta = dict(sigma=sigma, flipped0=flipped_fraction(W0, T))
    return wl


def cube_deform(cells: int = 64, seed: int = 3, jitter: float = 0.1,
                energy: str = SYM_DIRICHLET, rho: float = 10.0, max_iter: int = 1000,
                angle_deg: float = 45.0, shift_x: float = 0.3) -> Workload:
    """3D deformation: unit cube, cells^3 cubes, 6 tets each.

    Interior vertices are jittered uniformly by +-jitter cells (cube faces stay
    planar).  Bottom face z=0 is fixed; every top-face vertex is a handle, rotated
    by angle_deg about the z axis through (0.5, 0.5, 1) and then translated by
    shift_x in x.  W0 = rest pose with the handles snapped to their targets.
    Penalties mu_i = rho w_i with rho = 10: with rho = 3 the 64^3 cube keeps ~200
    tets flipped through 1000 iterations (the bound of the paper's convergence
    analysis is about 45 w_i for this energy at the rest state).
    """
    rng = np.random.default_rng(seed)
    V, T = cube_tets(cells)
    h = 1.0 / cells
    on_face = np.any((V < 0.5 * h) | (V > 1 - 0.5 * h), axis=1)
    inner = ~on_face
    V[inner] += rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 3))
    bottom = np.nonzero(V[:, 2] < 0.5 * h)[0]
    top = np.nonzero(V[:, 2] > 1 - 0.5 * h)[0]
    a = math.radians(angle_deg)
    R = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0, 0, 1.0]])
    c = np.array([0.5, 0.5, 1.0])
    top_pos = (V[top] - c) @ R.T + c + np.array([shift_x, 0.0, 0.0])
    pins = np.concatenate([bottom, top]).astype(np.int32)
    pin_pos = np.concatenate([V[bottom], top_pos])
    W0 = V.copy()
    W0[top] = top_pos
    wl = Workload(f"cube_deform_{cells}", V, T, pins, pin_pos, W0, energy, rho,
                  eps_abs=5e-10, eps_rel=5e-9, max_iter=max_iter)
    wl.meta = dict(flipped0=flipped_fraction(W0, T), n_handles=len(top))
    return wl


def bend_map(X: np.ndarray, radius: float = 2.0) -> np.ndarray:
    """Analytic bend T(x,y,z) = (R - (R-x) cos(z/R), y, (R-x) sin(z/R))."""
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return np.column_stack([radius - (radius - x) * np.cos(z / radius), y,
                            (radius - x) * np.sin(z / radius)])


def cube_handles(cells: int = 32, seed: int = 5, n_targets: int = 1000,
                 energy: str = SYM_DIRICHLET, rho: float = 3.0, lattice_start: int = 2,
                 lattice_step: int = 4, pre_bend: float = 0.0) -> Workload:
    """Differentiation workload: cube, bottom fixed, a lattice of top-face handles.

    Handles are the top-face vertices with lattice indices in
    {lattice_start, lattice_start + lattice_step, ...}^2 (64 for cells=32).  The
    handles' positions b (the parameters) start part-way along the bend map,
    b = rest + pre_bend (bend(rest) - rest), at rest by default; W0 is the rest
    pose (independent of b).  The loss targets are the bend map of n_targets seeded interior vertices.
    """
    rng = np.random.default_rng(seed)
    V, T = cube_tets(cells)
    k1 = cells + 1
    h = 1.0 / cells
    on_face = np.any((V < 0.5 * h) | (V > 1 - 0.5 * h), axis=1)
    inner = ~on_face
    V[inner] += rng.uniform(-0.1 * h, 0.1 * h, size=(inner.sum(), 3))
    bottom = np.nonzero(V[:, 2] < 0.5 * h)[0]
    lat = np.arange(lattice_start, cells, lattice_step)
    hi_, hj_ = np.meshgrid(lat, lat, indexing="ij")
    handles = ((hi_.ravel() * k1 + hj_.ravel()) * k1 + cells).astype(np.int32)
    pins = np.concatenate([bottom, handles]).astype(np.int32)
    pin_pos = V[pins].copy()
    hp = V[handles]
    pin_pos[len(bottom):] = hp + pre_bend * (bend_map(hp) - hp)
    n_targets = min(n_targets, int(inner.sum()))
    targets_idx = np.sort(rng.choice(np.nonzero(inner)[0], size=n_targets, replace=False))
    wl = Workload(f"cube_handles_{cells}", V, T, pins, pin_pos, V.copy(), energy, rho,
                  eps_abs=1e-6, eps_rel=1e-5, max_iter=200)
    wl.meta = dict(handles=handles, n_bottom=len(bottom), target_idx=targets_idx.astype(np.int32),
                   targets=bend_map(V[targets_idx]))
    return wl


def twist_bend_map(X: np.ndarray, twist: float = 4.0, radius: float = 2.0) -> np.ndarray:
    """Analytic target of the volume-correspondence workload: a twist by
    twist * z radians about the vertical axis through (0.5, 0.5), then the bend map."""
    x, y, z = X[:, 0] - 0.5, X[:, 1] - 0.5, X[:, 2]
    a = twist * z
    Y = np.column_stack([0.5 + x * np.cos(a) - y * np.sin(a), 0.5 + x * np.sin(a) + y * np.cos(a), z])
    return bend_map(Y, radius)


def volume_correspondence(cells: int = 32, seed: int = 6, twist: float = 4.0, radius: float = 2.0,
                          energy: str = SYM_GRADIENT, rho: float = 20.0, max_iter: int = 1000,
                          start: bool = True) -> Workload:
    """Volume correspondence (Sec. Results, "Volume Correspondence"): the interior of
    one closed surface mapped onto the interior of a second one whose boundary
    corresponds to it, with the boundary held on the second surface and the
    interior started from the minimizer of Tutte's energy (App. A).

    Synthetic stand-in for the paper's human and teddy-bear meshes: the unit cube
    (cells^3 cubes, 6 tets each, interior jittered by +-0.1 cell) is the first
    volume; every vertex on its boundary is pinned to its image under
    twist_bend_map (a twist by twist * z radians about the vertical axis through
    the centre, then a bend of radius `radius`), which carries the cube's boundary
    onto the second surface.  W0 is the Tutte map with that boundary (weights
    1 / |V_i - V_j|); on coarse meshes it folds some tets (0.07% at 8^3 cells), on
    fine ones it need not.  The symmetric gradient energy, as the paper uses for
    volume correspondence; eps_abs / eps_rel at the paper's defaults; mu_i = 20 w_i
    (with 10 w_i the 6^3 case oscillates flip-free above its tolerance; with 20 it
    converges at 6^3 to 16^3 within about 100 iterations).  Refuses a boundary
    map that inverts a tet whose four vertices are all pinned (no flip-free map
    would then exist).  start=False leaves W0 at the source positions with the
    boundary on the second surface (for callers that compute the Tutte start
    themselves).
    """
    rng = np.random.default_rng(seed)
    V, T = cube_tets(cells)
    h = 1.0 / cells
    on_face = np.any((V < 0.5 * h) | (V > 1 - 0.5 * h), axis=1)
    V[~on_face] += rng.uniform(-0.1 * h, 0.1 * h, size=((~on_face).sum(), 3))
    pins = np.nonzero(on_face)[0].astype(np.int32)
    pin_pos = twist_bend_map(V[pins], twist, radius)
    Wt = V.copy()
    Wt[pins] = pin_pos
    all_pinned = on_face[T].all(axis=1)
    if np.any(_signed_measure(Wt, T)[all_pinned] <= 0):
        raise ValueError("the boundary map inverts a tetrahedron whose vertices are all pinned")
    W0 = tutte_embedding(V, T, pins, pin_pos) if start else Wt
    wl = Workload(f"volume_correspondence_{cells}", V, T, pins, pin_pos, W0, energy, rho,
                  eps_abs=1e-6, eps_rel=1e-5, max_iter=max_iter)
    wl.meta = dict(flipped0=flipped_fraction(W0, T) if start else None, twist=twist, radius=radius)
    return wl


def batched_meshes(count: int = 256, seed: int = 4, m_min: int = 500, m_max: int = 50_000,
                   rho: float = 3.0, tol: float = 1e-5) -> list[Workload]:
    """Independent meshes for the batched solver.

    Sizes are drawn log-uniformly in [m_min, m_max] elements; even entries are
    jittered triangle grids (two corner vertices pinned), odd entries jittered
    cube tet meshes (bottom face pinned).  W0 is the rest pose plus Gaussian
    noise scaled so that a fraction drawn uniformly in [1%, 5%] of the elements
    starts flipped; the energy is symmetric Dirichlet or symmetric gradient at
    random.  Mesh j uses the seed 1000 + j.
    """
    top = np.random.default_rng(seed)
    sizes = np.exp(top.uniform(np.log(m_min), np.log(m_max), size=count))
    out = []
    for j in range(count):
        rng = np.random.default_rng(1000 + j)
        energy = SYM_DIRICHLET if rng.uniform() < 0.5 else SYM_GRADIENT
        frac = rng.uniform(0.01, 0.05)
        if j % 2 == 0:
            g = max(3, int(round(math.sqrt(sizes[j] / 2.0))) + 1)
            V, T = grid_triangles(g, g)
            h = 1.0 / (g - 1)
            bnd = np.zeros(V.shape[0], bool)
            bnd[_grid_boundary_cycle(g, g)] = True
            V[~bnd] += rng.uniform(-0.2 * h, 0.2 * h, size=((~bnd).sum(), 2))
            pins = np.array([0, (g - 1) * g], dtype=np.int32)
        else:
            c = max(2, int(round((sizes[j] / 6.0) ** (1.0 / 3.0))))
            V, T = cube_tets(c)
            h = 1.0 / c
            on_face = np.any((V < 0.5 * h) | (V > 1 - 0.5 * h), axis=1)
            V[~on_face] += rng.uniform(-0.1 * h, 0.1 * h, size=((~on_face).sum(), 3))
            pins = np.nonzero(V[:, 2] < 0.5 * h)[0].astype(np.int32)
        xi = rng.standard_normal(size=V.shape)
        xi[pins] = 0.0
        sigma = _noise_scale_for_flips(V, xi, T, frac, hi=2.0 * h)
        W0 = V + sigma * xi
        wl = Workload(f"batch_{j}", V, T, pins, V[pins].copy(), W0, energy, rho,
                      eps_abs=tol, eps_rel=10 * tol, max_iter=1000)
        wl.meta = dict(flipped0=flipped_fraction(W0, T), sigma=sigma)
        out.append(wl)
    return out


def by_name(name: str) -> Workload:
    """The five named workloads at full size."""
    if name == "uv_disk_48":
        return uv_disk()
    if name == "uv_heightfield_512":
        return uv_heightfield()
    if name == "cube_deform_64":
        return cube_deform()
    if name == "cube_handles_32":
        return cube_handles()
    if name == "volume_correspondence_32":
        return volume_correspondence()
    raise KeyError(name)
