"""ffa_energy_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a frozen or custom allocator, a pool that must not grow, a process
that only receives device buffers) cannot create a context, so this entry point
evaluates the energy of a map straight from device buffers, keeping its partial
sums in a fixed static device array.  It must agree with the context-based
ffa_energy (double precision local step) and with the FP64 oracle's energy to the
FP64 tolerance used elsewhere in these tests, on consecutive calls that share
that array.  This file is collected last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05200_gb300 import _native as N
    return torch, N, N.load()


def _cases():
    cube = wk.cube_deform(cells=5, seed=41)
    rng = np.random.default_rng(41)
    Wc = cube.V + 0.01 * rng.normal(size=cube.V.shape)
    surf = wk.uv_heightfield(grid=20, seed=42)
    Ws = surf.V[:, :2] + 0.002 * rng.normal(size=(surf.n, 2))
    return [(cube, Wc), (surf, Ws)]


def _noalloc_energy(torch, lib, wl, W, E_dev):
    dev = "cuda"
    V = torch.tensor(wl.V, dtype=torch.float64, device=dev)
    T = torch.tensor(wl.T, dtype=torch.int32, device=dev)
    Wd = torch.tensor(W, dtype=torch.float64, device=dev)
    code = 0 if wl.energy == "sd" else 1
    E_dev.fill_(float("nan"))
    st = lib.ffa_energy_noalloc(wl.n, wl.m, wl.d, wl.V.shape[1], C.c_void_p(V.data_ptr()),
                                C.c_void_p(T.data_ptr()), C.c_void_p(Wd.data_ptr()), code,
                                C.c_void_p(E_dev.data_ptr()), None)
    torch.cuda.synchronize()
    return st, float(E_dev.item())


def test_noalloc_energy_matches_context_energy_on_consecutive_calls():
    torch, N, lib = _setup()
    from paper_2107_05200_gb300.solver import Solver
    E_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    refs = []
    for wl, W in _cases():
        with Solver.from_workload(wl, precision="fp64") as sol:
            refs.append(sol.energy(W))
        E_oracle = admm.Oracle.from_workload(wl).energy(W)
        st, E = _noalloc_energy(torch, lib, wl, W, E_dev)
        assert st == 0 and math.isclose(E, E_oracle, rel_tol=RTOL), (wl.name, E, E_oracle)
    # two calls in a row per case, alternating sizes so stale partials would show
    for rep in range(2):
        for (wl, W), ref in zip(_cases(), refs):
            st, E = _noalloc_energy(torch, lib, wl, W, E_dev)
            assert st == 0, lib.ffa_last_error(None)
            assert math.isfinite(ref)
            assert math.isclose(E, ref, rel_tol=RTOL), (wl.name, rep, E, ref)


def test_noalloc_energy_flipped_and_limits():
    torch, N, lib = _setup()
    wl, W = _cases()[0]
    E_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    Wf = W.copy()
    Wf[:, 0] *= -1.0
    st, E = _noalloc_energy(torch, lib, wl, Wf, E_dev)
    assert st == 0 and E == math.inf
    dummy = C.c_void_p(E_dev.data_ptr())
    st = lib.ffa_energy_noalloc(10, 16777217, 3, 3, dummy, dummy, dummy, 0, dummy, None)
    assert st == 1
    assert b"16,777,216" in lib.ffa_last_error(None)
    st = lib.ffa_energy_noalloc(10, 5, 4, 3, dummy, dummy, dummy, 0, dummy, None)
    assert st == 1


def test_noalloc_energy_reports_invalid_meshes_as_nan():
    """An index outside [0, n) (too large or negative) is caught before any load through
    it, and a zero-measure source element is not evaluated: both give NaN, which a
    flipped map of a valid mesh (+inf) never does.  A valid call afterwards is exact."""
    torch, N, lib = _setup()
    wl, W = _cases()[0]
    E_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    for bad in (wl.n + 5, -1):
        T = wl.T.copy()
        T[3, 2] = bad
        st, E = _noalloc_energy(torch, lib, wk.Workload("bad", wl.V, T, wl.pins, wl.pin_pos, W, wl.energy), W, E_dev)
        assert st == 0 and math.isnan(E), bad
    T = wl.T.copy()
    T[7, 1] = T[7, 0]          # two equal vertices: zero volume
    st, E = _noalloc_energy(torch, lib, wk.Workload("degenerate", wl.V, T, wl.pins, wl.pin_pos, W, wl.energy), W,
                            E_dev)
    assert st == 0 and math.isnan(E)
    st, E = _noalloc_energy(torch, lib, wl, W, E_dev)
    assert st == 0 and math.isclose(E, admm.Oracle.from_workload(wl).energy(W), rel_tol=RTOL)
