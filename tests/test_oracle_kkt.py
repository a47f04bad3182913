"""The oracle's converged iterates are KKT points of the split problem (Sec. 5,
eq. kkt), checked condition by condition with the multiplier M_i = mu_i Lambda_i:

  * w_i grad f(P_i) = U_i^T M_i, unsymmetrized (the P step only enforces the
    symmetric part at every iteration; at a KKT point U_i^T M_i is symmetric);
  * stationarity of U_i on SO(d) (the second condition): U_i^T M_i P_i symmetric;
  * (G W)_i = U_i P_i;
  * stationarity in W, which the conditions imply through the W step: G^T M
    vanishes at the free vertices.

Each run is driven to tolerances far below the paper's (eps_abs 1e-12,
eps_rel 1e-11) so that the residuals reach the level of the iterates' own
convergence.  No GPU is used."""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

CASES = {
    "disk_sd": lambda: wk.uv_disk(grid=12, seed=5, rho=3.0),
    "disk_sg": lambda: wk.uv_disk(grid=12, seed=5, rho=3.0, energy="sg"),
    "cube_sd": lambda: wk.cube_deform(cells=3, seed=5, rho=10.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_converged_iterates_satisfy_the_kkt_conditions(case):
    wl = CASES[case]()
    o = admm.Oracle.from_workload(wl, eps_abs=1e-12, eps_rel=1e-11)
    s, st = o.run(wl.W0, 3000)
    assert st.converged and st.n_flipped == 0
    tr = lambda X: np.transpose(X, (0, 2, 1))
    M = o.mu[:, None, None] * s.Lam
    wgrad = o.w[:, None, None] * admm.grad_f(s.P, o.energy_name)
    assert np.abs(wgrad - tr(s.U) @ M).max() <= 1e-8 * np.abs(wgrad).max()
    A = tr(s.U) @ M @ s.P
    assert np.abs(A - tr(A)).max() <= 1e-8 * np.abs(A).max()
    assert np.abs(s.J - s.U @ s.P).max() <= 1e-8
    free = np.setdiff1d(np.arange(o.n), wl.pins)
    GtM = admm.gradient_adjoint(o.g, o.T, M, o.n)[free]
    scale = admm.gradient_adjoint(o.g, o.T, np.abs(M), o.n)[free]
    assert np.abs(GtM).max() <= 1e-7 * np.abs(scale).max()
    # the multiplier is not trivially zero: the map is deformed
    assert np.abs(M).max() > 1e-4
