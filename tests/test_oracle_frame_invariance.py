"""Pin of the oracle's Jacobian convention and of its local steps through a
symmetry. Rotate the source mesh by Q in SO(d): the hat-function gradients turn
with it, so J_i = (G W)_i becomes Q J_i, with rows indexing source directions and
column k the gradient of target coordinate k (Supplemental, "Computing the
Jacobian Map"). L = sum_i mu_i G_i^T G_i does not change. Because f is rotation
invariant, the whole iteration then maps U_i to Q U_i and Lambda_i to Q Lambda_i
and keeps W and P as they are (J = U P with U on the source side). A transposed
Jacobian, a U applied on the wrong side, or a frame-dependent step breaks it. An
intrinsic (surface) mesh moved rigidly in R^3 gives the same iterates outright."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def _run(V, T, pins, pin_pos, W0, energy, K=12):
    o = admm.Oracle(V, T, pins, pin_pos, energy, rho=3.0)
    s = o.init(W0)
    out = [s]
    for _ in range(K):
        s, _ = o.step(s)
        out.append(s)
    return out


def _case(d):
    if d == 2:
        wl = wk.uv_disk(grid=9, seed=81, rho=3.0)
        W0 = 1.3 * (wl.V - 0.5)
        W0[wl.pins] = wl.pin_pos
        return wl.V, wl.T, wl.pins, wl.pin_pos, W0
    wl = wk.cube_deform(cells=3, seed=82)
    return wl.V, wl.T, wl.pins, wl.pin_pos, wl.W0


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("energy", ["sd", "sg", "sa"])
def test_rotating_the_source_rotates_u_and_lambda_only(d, energy):
    V, T, pins, pin_pos, W0 = _case(d)
    if d == 2:
        a = 0.7
        Q = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    else:
        Q = Rotation.from_rotvec([0.4, -0.9, 0.3]).as_matrix()
    ref = _run(V, T, pins, pin_pos, W0, energy)
    rot = _run(V @ Q.T, T, pins, pin_pos, W0, energy)
    for s0, s1 in zip(ref, rot):
        scale = np.abs(s0.W).max()
        np.testing.assert_allclose(s1.W, s0.W, rtol=0, atol=1e-10 * scale)
        np.testing.assert_allclose(s1.J, Q @ s0.J, rtol=0, atol=1e-9 * np.abs(s0.J).max())
        np.testing.assert_allclose(s1.P, s0.P, rtol=0, atol=1e-9 * np.abs(s0.P).max())
        np.testing.assert_allclose(s1.U, Q @ s0.U, rtol=0, atol=1e-9)
        np.testing.assert_allclose(s1.Lam, Q @ s0.Lam, rtol=0, atol=1e-9 * max(1.0, np.abs(s0.Lam).max()))


def test_surface_mesh_moved_rigidly_in_space_gives_the_same_iterates():
    V2, T = wk.grid_triangles(6, 5)
    rng = np.random.default_rng(83)
    V2 = V2 + rng.uniform(-0.05, 0.05, V2.shape)
    R = Rotation.from_rotvec([0.3, -0.7, 0.2]).as_matrix()
    Vs = np.column_stack([V2, np.zeros(len(V2))]) @ R.T + np.array([0.1, 0.2, 0.3])
    R2 = Rotation.from_rotvec([-1.1, 0.5, 0.8]).as_matrix()
    Vs2 = Vs @ R2.T - np.array([0.4, 0.0, 0.2])
    pins = np.array([0, 5], dtype=np.int64)
    W0 = V2 * np.array([1.2, 0.8]) + 0.02 * rng.normal(size=V2.shape)
    pin_pos = W0[pins]
    a = _run(Vs, T, pins, pin_pos, W0, "sg")
    b = _run(Vs2, T, pins, pin_pos, W0, "sg")
    for s0, s1 in zip(a, b):
        np.testing.assert_allclose(s1.W, s0.W, rtol=0, atol=1e-11)
        np.testing.assert_allclose(s1.U, s0.U, rtol=0, atol=1e-9)
        np.testing.assert_allclose(s1.P, s0.P, rtol=0, atol=1e-9)
