"""Failure detection of the W step's bounded device waits, made to run out on purpose
without faulting the GPU.

With the dynamic schedule each block of a triangular pass polls its queue slot
until a finished supernode fills it.  ffa_set_wait_limit(0) makes a wait give up
at its first empty poll, which on a multi-level elimination tree happens in the
first pass (blocks claim slots beyond the initially ready tasks at launch): the
kernel sets its error flag, every block exits, and ffa_iterate must return
FFA_ERR_TIMEOUT with the context still usable.  The GPU must keep answering, the
same context must solve correctly once the default limit is restored, and a fresh
context must match the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu

DEFAULT_POLLS = 1 << 22


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("schedule", [1, 2])
def test_wait_limit_runs_out_and_the_context_recovers(schedule):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05200_gb300._native import FFAError
    from paper_2107_05200_gb300.solver import Solver

    wl = wk.cube_deform(cells=10, seed=41)
    iters = 5
    o = admm.Oracle.from_workload(wl)
    s = o.init(wl.W0)
    for _ in range(iters):
        s, _ = o.step(s)

    with Solver.from_workload(wl, precision="fp64", check_every=1, schedule=schedule) as sol:
        assert sol.info()["n_levels"] >= 4
        sol.init(wl.W0)
        sol.set_wait_limit(0)
        with pytest.raises(FFAError, match="TIMEOUT"):
            sol.iterate(iters, stop_at_tol=False)
        # the device still answers
        x = torch.arange(1000, device="cuda", dtype=torch.float64)
        assert float(x.sum().item()) == 499500.0
        torch.cuda.synchronize()
        # the same context with the default limit restored, from the start again
        sol.set_wait_limit(DEFAULT_POLLS)
        sol.init(wl.W0)
        sol.iterate(iters, stop_at_tol=False)
        W_same = sol.W()
    with pytest.raises(FFAError, match="INVALID_ARG"):
        with Solver.from_workload(wl, precision="fp64") as sol:
            sol.set_wait_limit(-1)
    with Solver.from_workload(wl, precision="fp64", check_every=1, schedule=schedule) as fresh:
        fresh.init(wl.W0)
        fresh.iterate(iters, stop_at_tol=False)
        W_fresh = fresh.W()
    assert _rel(W_fresh, s.W) < 1e-8
    assert _rel(W_same, s.W) < 1e-8
