"""The seeded input generators build the workloads their recipes state.

The paper's meshes are not available, so the parity cases and the benchmark run
on synthetic stand-ins (the 2D disk and heightfield parametrizations of Sec. 7,
the tetrahedral deformations, the volume correspondence of Sec. Results).  These
tests check each generator's output against its recipe, recomputing the geometry
the recipe names (rotation, bend, twist, circle placement, Tutte averages)
independently of the generator: sizes, which vertices are pinned and where, the
jitter bounds, the orientation of the source elements, the flipped fraction of
the initial map, and that no element of an initial map sits at the flip
threshold, so that no flip decision is left to rounding.  No GPU is used.
"""
import math

import numpy as np
import pytest

from paper_2107_05200_gb300 import workloads as wk


def _measure(X, T):
    """Signed area / volume of each element, written out here."""
    if T.shape[1] == 3:
        a, b, c = X[T[:, 0]], X[T[:, 1]], X[T[:, 2]]
        return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    a, b, c, e = (X[T[:, k]] for k in range(4))
    return np.linalg.det(np.stack([b - a, c - a, e - a], axis=1)) / 6.0


def _flipped(W, T):
    return int(np.sum(_measure(W, T) <= 0.0))


def _faces_conform(T):
    """Every facet of a simplicial mesh of a ball is shared by at most two
    elements; returns the number of boundary facets (those used once)."""
    k = T.shape[1]
    F = np.concatenate([np.delete(T, j, axis=1) for j in range(k)], 0)
    F = np.sort(F, axis=1)
    _, cnt = np.unique(F, axis=0, return_counts=True)
    assert cnt.max() <= 2
    return int(np.sum(cnt == 1))


def _neighbours(T, n):
    k = T.shape[1]
    nb = [set() for _ in range(n)]
    for a in range(k):
        for b in range(k):
            if a != b:
                for u, v in zip(T[:, a], T[:, b]):
                    nb[u].add(int(v))
    return nb


# --------------------------------------------------------------------------
# 2D: the disk parametrization (48 x 48 grid)
# --------------------------------------------------------------------------

def test_uv_disk_recipe():
    wl = wk.uv_disk()
    g = 48
    h = 1.0 / (g - 1)
    assert (wl.n, wl.m, wl.d, wl.d_in, wl.d_out) == (2304, 4418, 2, 2, 2)
    assert (wl.energy, wl.rho, wl.max_iter) == ("sd", 1.0, 500)
    assert math.isclose(wl.eps_abs, 1e-6) and math.isclose(wl.eps_rel, 1e-5)
    # the grid: boundary vertices on the square's boundary, interior ones within +-0.2 cells
    i, j = np.divmod(np.arange(wl.n), g)
    grid = np.stack([i / (g - 1), j / (g - 1)], 1)
    on_bnd = (i == 0) | (i == g - 1) | (j == 0) | (j == g - 1)
    assert set(wl.pins.tolist()) == set(np.flatnonzero(on_bnd).tolist()) and len(wl.pins) == 4 * (g - 1)
    np.testing.assert_array_equal(wl.V[on_bnd], grid[on_bnd])
    dev = np.abs(wl.V[~on_bnd] - grid[~on_bnd])
    assert dev.max() <= 0.2 * h and dev.max() > 0.15 * h
    assert np.all(_measure(wl.V, wl.T) > 0.0)
    assert math.isclose(_measure(wl.V, wl.T).sum(), 1.0, rel_tol=1e-12)
    # no triangle has all three vertices pinned
    assert not np.any(on_bnd[wl.T].all(axis=1))
    # pins on the unit circle, counter-clockwise, spaced by source arc length
    r = np.linalg.norm(wl.pin_pos, axis=1)
    np.testing.assert_allclose(r, 1.0, atol=1e-15)
    ang = np.unwrap(np.arctan2(wl.pin_pos[:, 1], wl.pin_pos[:, 0]))
    ang -= ang[0]
    assert np.all(np.diff(ang) > 0)
    Vb = wl.V[wl.pins]
    seg = np.linalg.norm(np.roll(Vb, -1, axis=0) - Vb, axis=1)
    np.testing.assert_allclose(np.diff(ang), 2 * math.pi * seg[:-1] / seg.sum(), atol=1e-12)
    # W0: the Tutte map (each interior vertex the 1/|V_i - V_j|-weighted average of
    # its neighbours) plus noise on the interior, 3% of the triangles flipped
    np.testing.assert_array_equal(wl.W0[wl.pins], wl.pin_pos)
    Wt = wk.tutte_embedding(wl.V, wl.T, wl.pins, wl.pin_pos)
    nb = _neighbours(wl.T, wl.n)
    for v in np.flatnonzero(~on_bnd)[::37]:
        js = sorted(nb[v])
        wts = 1.0 / np.linalg.norm(wl.V[js] - wl.V[v], axis=1)
        np.testing.assert_allclose(Wt[v], wts @ Wt[js] / wts.sum(), atol=1e-12)
    assert _flipped(Wt, wl.T) == 0                      # Tutte's theorem: convex boundary, no flips
    assert _flipped(wl.W0, wl.T) == math.ceil(0.03 * wl.m)
    # off the flip threshold: every |det| at least 1e-6 of the unperturbed one
    assert np.all(np.abs(_measure(wl.W0, wl.T)) >= 1e-6 * np.abs(_measure(Wt, wl.T)))


# --------------------------------------------------------------------------
# surface: the heightfield parametrization (512 x 512 grid)
# --------------------------------------------------------------------------

def test_uv_heightfield_recipe():
    wl = wk.uv_heightfield()
    g = 512
    assert (wl.n, wl.m, wl.d, wl.d_in, wl.d_out) == (262144, 522242, 2, 3, 2)
    assert (wl.energy, wl.rho) == ("sg", 10.0)
    assert math.isclose(wl.eps_abs, 1e-5) and math.isclose(wl.eps_rel, 1e-4)
    i, j = np.divmod(np.arange(wl.n), g)
    x, y = i / (g - 1), j / (g - 1)
    np.testing.assert_array_equal(wl.V[:, 0], x)
    np.testing.assert_array_equal(wl.V[:, 1], y)
    np.testing.assert_allclose(wl.V[:, 2], 0.3 * np.sin(3 * x) * np.cos(2 * y), atol=1e-15)
    # two pins at the projected positions of (0, 0) and (1, 0)
    np.testing.assert_array_equal(wl.V[wl.pins, :2], [[0.0, 0.0], [1.0, 0.0]])
    np.testing.assert_array_equal(wl.pin_pos, wl.V[wl.pins, :2])
    np.testing.assert_array_equal(wl.W0[wl.pins], wl.pin_pos)
    # the projection plus noise: 5.0 +- 0.5 % flipped, none at the threshold
    P2 = wl.V[:, :2]
    assert np.all(_measure(P2, wl.T) > 0.0)
    f = _flipped(wl.W0, wl.T) / wl.m
    assert 0.05 <= f <= 0.055
    assert np.all(np.abs(_measure(wl.W0, wl.T)) >= 1e-6 * _measure(P2, wl.T))


# --------------------------------------------------------------------------
# 3D: the benchmark cube (64^3 cells, 6 tets each)
# --------------------------------------------------------------------------

def test_cube_deform_recipe():
    wl = wk.cube_deform()
    c = 64
    h = 1.0 / c
    assert (wl.n, wl.m, wl.d, wl.d_in) == (274625, 1572864, 3, 3)
    assert (wl.energy, wl.rho, wl.eps_abs, wl.eps_rel, wl.max_iter) == ("sd", 10.0, 5e-10, 5e-9, 1000)
    lat = np.stack(np.meshgrid(*(np.arange(c + 1),) * 3, indexing="ij"), -1).reshape(-1, 3) / c
    on_face = np.any((lat == 0.0) | (lat == 1.0), axis=1)
    np.testing.assert_array_equal(wl.V[on_face], lat[on_face])          # faces stay planar
    dev = np.abs(wl.V[~on_face] - lat[~on_face])
    assert dev.max() <= 0.1 * h and dev.max() > 0.09 * h
    vol = _measure(wl.V, wl.T)
    assert np.all(vol > 0.0)
    assert math.isclose(vol.sum(), 1.0, rel_tol=1e-12)
    # pins: the bottom face at rest, every top-face vertex rotated by 45 degrees
    # about the vertical axis through (0.5, 0.5, 1) and shifted by 0.3 in x
    bottom = np.flatnonzero(wl.V[:, 2] == 0.0)
    top = np.flatnonzero(wl.V[:, 2] == 1.0)
    assert len(bottom) == len(top) == (c + 1) ** 2
    np.testing.assert_array_equal(np.sort(wl.pins), np.sort(np.concatenate([bottom, top])))
    pos = dict(zip(wl.pins.tolist(), wl.pin_pos))
    np.testing.assert_array_equal(np.array([pos[v] for v in bottom]), wl.V[bottom])
    s = 1.0 / math.sqrt(2.0)
    x, y = wl.V[top, 0] - 0.5, wl.V[top, 1] - 0.5
    want = np.stack([0.5 + s * (x - y) + 0.3, 0.5 + s * (x + y), np.ones_like(x)], 1)
    np.testing.assert_allclose(np.array([pos[v] for v in top]), want, atol=1e-15)
    # W0: the rest pose with the handles snapped; only tets touching the top face invert
    rest = np.setdiff1d(np.arange(wl.n), top)
    np.testing.assert_array_equal(wl.W0[rest], wl.V[rest])
    np.testing.assert_array_equal(wl.W0[top], np.array([pos[v] for v in top]))
    fl = _measure(wl.W0, wl.T) <= 0.0
    assert 0.001 < fl.mean() < 0.005
    is_top = np.zeros(wl.n, bool)
    is_top[top] = True
    assert np.all(is_top[wl.T[fl]].any(axis=1))


@pytest.mark.parametrize("cells", [3, 8])
def test_kuhn_split_is_a_conforming_mesh_of_the_cube(cells):
    """6 tets per cell sharing each cell's main diagonal: every facet is shared by
    at most two tets, and the boundary is the cube's 6 faces, 2 triangles per cell
    square."""
    V, T = wk.cube_tets(cells)
    assert T.shape == (6 * cells ** 3, 4) and V.shape == ((cells + 1) ** 3, 3)
    vol = _measure(V, T)
    np.testing.assert_allclose(vol, 1.0 / (6 * cells ** 3), rtol=1e-12)
    assert _faces_conform(T) == 12 * cells ** 2


# --------------------------------------------------------------------------
# differentiation: the handle cube (32^3 cells)
# --------------------------------------------------------------------------

def test_cube_handles_recipe():
    wl = wk.cube_handles()
    c = 32
    h = 1.0 / c
    assert (wl.n, wl.m, wl.max_iter) == (35937, 196608, 200)
    bottom = np.flatnonzero(wl.V[:, 2] == 0.0)
    nb = wl.meta["n_bottom"]
    assert nb == len(bottom) == (c + 1) ** 2
    handles = wl.pins[nb:]
    assert len(handles) == 64
    lattice = set(range(2, 31, 4))
    got = {(round(wl.V[v, 0] / h), round(wl.V[v, 1] / h)) for v in handles}
    assert got == {(a, b) for a in lattice for b in lattice}
    assert np.all(wl.V[handles, 2] == 1.0)
    np.testing.assert_array_equal(wl.pin_pos, wl.V[wl.pins])         # handles start at rest
    np.testing.assert_array_equal(wl.W0, wl.V)
    # 1000 distinct interior targets, moved by the bend of radius 2
    idx = wl.meta["target_idx"]
    assert len(idx) == len(set(idx.tolist())) == 1000
    X = wl.V[idx]
    assert np.all((X > 0.0) & (X < 1.0))
    R = 2.0
    want = np.stack([R - (R - X[:, 0]) * np.cos(X[:, 2] / R), X[:, 1], (R - X[:, 0]) * np.sin(X[:, 2] / R)], 1)
    np.testing.assert_allclose(wl.meta["targets"], want, atol=1e-15)


# --------------------------------------------------------------------------
# the volume correspondence stand-in
# --------------------------------------------------------------------------

def test_volume_correspondence_recipe():
    cells = 6
    wl = wk.volume_correspondence(cells=cells)
    on_face = np.any((wl.V == 0.0) | (wl.V == 1.0), axis=1)
    np.testing.assert_array_equal(np.sort(wl.pins), np.flatnonzero(on_face))
    # the boundary on the second surface: a twist by 4z about the axis through
    # (0.5, 0.5), then the bend of radius 2
    X = wl.V[wl.pins]
    a = 4.0 * X[:, 2]
    x, y = X[:, 0] - 0.5, X[:, 1] - 0.5
    tx, ty = 0.5 + x * np.cos(a) - y * np.sin(a), 0.5 + x * np.sin(a) + y * np.cos(a)
    R = 2.0
    want = np.stack([R - (R - tx) * np.cos(X[:, 2] / R), ty, (R - tx) * np.sin(X[:, 2] / R)], 1)
    np.testing.assert_allclose(wl.pin_pos, want, atol=1e-14)
    # the start: the Tutte map with that boundary
    np.testing.assert_allclose(wl.W0[wl.pins], wl.pin_pos, atol=0)
    nb = _neighbours(wl.T, wl.n)
    for v in np.flatnonzero(~on_face):
        js = sorted(nb[v])
        wts = 1.0 / np.linalg.norm(wl.V[js] - wl.V[v], axis=1)
        np.testing.assert_allclose(wl.W0[v], wts @ wl.W0[js] / wts.sum(), atol=1e-12)
    assert (wl.energy, wl.rho) == ("sg", 20.0)


# --------------------------------------------------------------------------
# the batch: 256 meshes, log-uniform sizes, half 2D, half 3D
# --------------------------------------------------------------------------

def test_batch_sizes_are_log_uniform_between_500_and_50k():
    from scipy import stats
    lo, hi = math.log(500), math.log(50_000)
    sizes = np.exp(np.random.default_rng(4).uniform(lo, hi, size=256))
    ks = stats.kstest((np.log(sizes) - lo) / (hi - lo), "uniform")
    assert ks.pvalue > 0.01


def test_batched_mesh_recipe():
    count = 16                       # the first meshes of the 256-mesh batch (same seeds)
    wls = wk.batched_meshes(count=count)
    sizes = np.exp(np.random.default_rng(4).uniform(math.log(500), math.log(50_000), size=256))[:count]
    energies = set()
    for j, (wl, s) in enumerate(zip(wls, sizes)):
        assert wl.d == (2 if j % 2 == 0 else 3) and wl.d_in == wl.d
        assert 0.6 * s <= wl.m <= 1.5 * s
        assert np.all(_measure(wl.V, wl.T) > 0.0)
        assert math.isclose(_measure(wl.V, wl.T).sum(), 1.0, rel_tol=1e-12)
        if wl.d == 2:
            np.testing.assert_array_equal(wl.V[wl.pins], [[0.0, 0.0], [1.0, 0.0]])
        else:
            np.testing.assert_array_equal(np.sort(wl.pins), np.flatnonzero(wl.V[:, 2] == 0.0))
        np.testing.assert_array_equal(wl.pin_pos, wl.V[wl.pins])
        np.testing.assert_array_equal(wl.W0[wl.pins], wl.V[wl.pins])
        f = _flipped(wl.W0, wl.T) / wl.m
        assert 0.01 <= f <= 0.055, (j, f)
        assert np.all(np.abs(_measure(wl.W0, wl.T)) >= 1e-6 * _measure(wl.V, wl.T))
        assert wl.rho == 3.0 and math.isclose(wl.eps_abs, 1e-5) and math.isclose(wl.eps_rel, 1e-4)
        energies.add(wl.energy)
    assert energies == {"sd", "sg"}
