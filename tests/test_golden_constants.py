"""The constants the paper prints for its initialization and penalty schedule
(tests/golden/printed_constants.txt, each line with its citation) against the
oracle, and against the C library's default parameters (no GPU needed)."""
import ctypes as C
import math
import os

import numpy as np
import pytest

from oracle import admm
from oracle import schedule as osched

HERE = os.path.dirname(os.path.abspath(__file__))
EPS_M = 2.0 ** -52


def _constants():
    out = {}
    with open(os.path.join(HERE, "golden", "printed_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, value = line.split()[:2]
            out[key] = float(value)
    return out


K = _constants()


@pytest.mark.parametrize("energy,key", [("sg", "init_clamp_exponent_sg"), ("sd", "init_clamp_exponent_sd")])
def test_polar_init_clamps_and_flips_with_the_printed_epsilon(energy, key):
    eps = EPS_M ** K[key]
    J = np.array([[[1.0, 0.0], [0.0, 1e-12]],        # a tiny singular value: raised to eps
                  [[2.0, 0.0], [0.0, -1.0]],         # flipped: Sigma = eps I, det U = 1
                  [[1.5, 0.2], [0.1, 0.9]]])         # regular: the polar decomposition itself
    U, P = admm.polar_init(J, energy)
    s0 = np.linalg.eigvalsh(P[0])
    assert math.isclose(s0.min(), eps, rel_tol=1e-12) and math.isclose(s0.max(), 1.0, rel_tol=1e-12)
    np.testing.assert_allclose(P[1], eps * np.eye(2), rtol=1e-12)
    assert math.isclose(np.linalg.det(U[1]), 1.0, rel_tol=1e-12)
    np.testing.assert_allclose(U[2] @ P[2], J[2], atol=1e-14)
    o = admm.Oracle(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[0, 1, 2]]), np.array([0]),
                    np.zeros((1, 2)), energy)
    s = o.init(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]))
    assert np.all(s.Lam == K["init_lambda"])


def test_rescaling_rule_and_events():
    assert osched.RESCALE_RHO == K["rescale_rho"]
    mu = np.array([1.0, 1.0, 1.0])
    Lam = np.ones((3, 2, 2))
    e_prim = np.array([10.0, 1.0, 1.0])
    e_dual = np.array([1.0, 10.0, 1.0])
    new, Lam2 = osched.rescale(mu, Lam, e_prim, e_dual, mu_lo=np.zeros(3))
    step = K["rescale_rho"] * K["rescale_step_over_rho"]
    np.testing.assert_allclose(new, [step, 1.0 / step, 1.0])
    np.testing.assert_allclose(Lam2[:, 0, 0], [1.0 / step, step, 1.0])   # mu_i Lambda_i unchanged
    # never below mu_min / 2: the caller passes that bound as mu_lo
    new, _ = osched.rescale(mu, Lam, e_dual, e_prim, mu_lo=np.full(3, 0.9))
    assert new.min() >= 0.9
    # events: the first initial_rescales iterations, then every
    # floor(period_base * period_ratio^p) with p the events so far
    want, k, p = list(range(1, int(K["initial_rescales"]) + 1)), int(K["initial_rescales"]), int(K["initial_rescales"])
    while True:
        k += int(math.floor(K["period_base"] * K["period_ratio"] ** p))
        if k > 2000:
            break
        want.append(k)
        p += 1
    assert osched.rescale_iterations(2000) == want


def test_f_cap_and_b_factor():
    P = np.broadcast_to(np.eye(3), (1, 3, 3)).copy()
    for energy in ("sd", "sg"):
        F = osched.lipschitz_F(np.array([1e12]), energy, 3)
        assert math.isclose(F[0] ** 2, EPS_M ** K["f2_cap_exponent"], rel_tol=1e-12)
        # B_i = sqrt(b_factor (1 + |grad f|^2)): at P = I the gradient of both energies vanishes
        B = math.sqrt(K["b_factor"] * (1.0 + 0.0))
        w = np.array([0.7])
        F1 = osched.lipschitz_F(np.array([B]), energy, 3)
        mu = osched.mu_min(P, w, energy)
        g, e = K["gamma"], K["epsilon"]
        want = 0.5 * (-(w - 2 * e) + np.sqrt((w - 2 * e) ** 2 + 16 * g * w * w * F1 * F1))
        np.testing.assert_allclose(mu, want, rtol=1e-14)


def test_library_defaults_match():
    from paper_2107_05200_gb300 import _native
    try:
        lib = _native.load()
    except RuntimeError:
        pytest.skip("libffadmm.so is not built")
    p = _native.Params()
    assert lib.ffa_default_params(C.byref(p)) == 0
    assert p.rescale_rho == K["rescale_rho"]
    assert p.penalty_schedule == 0
    assert p.eps_abs == K["eps_abs_default"] and p.eps_rel == K["eps_rel_default"]


def test_termination_tolerances():
    """The oracle's default tolerances are the printed ones for most examples; the 3D deformation
    workload takes the printed deformation values; the other workloads keep the printed ratio
    eps_rel / eps_abs = 10 for the tolerance their configuration states."""
    import inspect
    from paper_2107_05200_gb300 import workloads as wk
    sig = inspect.signature(admm.Oracle.__init__).parameters
    assert sig["eps_abs"].default == K["eps_abs_default"]
    assert sig["eps_rel"].default == K["eps_rel_default"]
    cube = wk.cube_deform(cells=2)
    assert cube.eps_abs == K["eps_abs_deformation"] and cube.eps_rel == K["eps_rel_deformation"]
    assert K["eps_rel_default"] / K["eps_abs_default"] == pytest.approx(10.0)
    assert K["eps_rel_deformation"] / K["eps_abs_deformation"] == pytest.approx(10.0)
    disk = wk.uv_disk(grid=8)
    assert disk.eps_rel / disk.eps_abs == pytest.approx(10.0)
