"""The Python binding's marshalling on a machine without a GPU: element counts
are checked before a pointer reaches the library (an undersized array would be
read or written past its end), and output buffers that the library cannot write
in place are refused rather than converted (a converted copy would receive the
results and drop them)."""
import numpy as np
import pytest

from paper_2107_05200_gb300 import solver as S


def test_input_counts_and_conversion():
    p, keep = S._ptr(np.arange(6, dtype=np.int64).reshape(2, 3), np.float64, 6, "W")
    assert keep.dtype == np.float64 and keep.flags.c_contiguous and p.value == keep.ctypes.data
    with pytest.raises(ValueError, match="W has 5 entries, the call reads 6"):
        S._ptr(np.zeros(5), np.float64, 6, "W")
    assert S._ptr(None, np.float64, 6, "W") == (None, None)
    torch = pytest.importorskip("torch")
    t = torch.arange(6, dtype=torch.float32).reshape(3, 2).t()   # float32, not contiguous
    p, keep = S._ptr(t, np.float64, 6, "W")
    assert keep.dtype == torch.float64 and keep.is_contiguous() and p.value == keep.data_ptr()
    with pytest.raises(ValueError):
        S._ptr(torch.zeros(7, dtype=torch.float64), np.float64, 6, "W")


def test_outputs_are_written_in_place_or_refused():
    a = np.zeros((3, 2))
    assert S._out(a, 6, "out").value == a.ctypes.data
    for bad in (np.zeros((3, 2), np.float32), np.zeros((2, 3)).T, np.zeros(5)):
        with pytest.raises(ValueError):
            S._out(bad, 6, "out")
    ro = np.zeros(6)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        S._out(ro, 6, "out")
    with pytest.raises(TypeError):
        S._out([0.0] * 6, 6, "out")
    torch = pytest.importorskip("torch")
    t = torch.zeros(3, 2, dtype=torch.float64)
    assert S._out(t, 6, "out").value == t.data_ptr()
    for bad in (torch.zeros(3, 2), torch.zeros(2, 3, dtype=torch.float64).t(), torch.zeros(5, dtype=torch.float64)):
        with pytest.raises(ValueError):
            S._out(bad, 6, "out")


class _NoLib:
    """Stands in for the loaded library: any call through it fails the test, so
    a refusal must come from the binding before the library is reached."""

    def __getattr__(self, name):
        raise AssertionError(f"the library was called ({name}) with an argument the binding should refuse")


def _solver(n=5, m=4, d=2, n_pin=2):
    s = object.__new__(S.Solver)
    s._lib, s._ctx = _NoLib(), None
    s.n, s.m, s.d, s.d_in, s.n_pin = n, m, d, d, n_pin
    return s


def test_solver_methods_check_sizes_before_the_library():
    s = _solver()
    with pytest.raises(ValueError):
        s.init(np.zeros((4, 2)))
    with pytest.raises(ValueError):
        s.set_handles(np.zeros((3, 2)))
    with pytest.raises(ValueError):
        s.energy(np.zeros((5, 3)))
    with pytest.raises(ValueError):
        s.gradient(np.zeros((5, 2)), out=np.zeros((5, 2), np.float32))
    with pytest.raises(ValueError):
        s.W(np.zeros((4, 2)))
    with pytest.raises(ValueError):
        s.set_state(np.zeros((5, 2)), np.zeros((4, 2, 2)), np.zeros((4, 2, 2)), np.zeros((3, 2, 2)))
    with pytest.raises(ValueError):
        s.backward_unrolled(np.zeros((5, 2)), out=np.zeros((3, 2)))


def test_batch_methods_check_counts_before_the_library():
    b = object.__new__(S.BatchSolver)
    b._lib, b._b, b.k, b.n, b.d = _NoLib(), None, 2, [4, 5], [2, 3]
    with pytest.raises(ValueError, match="1 initial maps for 2 meshes"):
        b.init([np.zeros((4, 2))])
    with pytest.raises(ValueError):
        b.init([np.zeros((4, 2)), np.zeros((5, 2))])
    with pytest.raises(ValueError):
        b.W(1, out=np.zeros((5, 2)))


class _RecordingLib:
    """Stands in for the loaded library: records each call and reports success."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append((name, args))
            return 0
        return fn


@pytest.mark.parametrize("d,d_in,n_pin", [(2, 2, 2), (2, 3, 2), (3, 3, 4), (2, 2, 0)])
def test_valid_arguments_reach_the_library(d, d_in, n_pin):
    """Every wrapped call with arrays of the documented shapes (numpy and torch
    CPU tensors) passes the binding's checks, and an output that is already a
    contiguous float64 buffer is handed over in place."""
    n, m = 7, 5
    s = object.__new__(S.Solver)
    lib = _RecordingLib()
    s._lib, s._ctx = lib, None
    s.n, s.m, s.d, s.d_in, s.n_pin = n, m, d, d_in, max(n_pin, 1)
    W = np.zeros((n, d))
    s.set_handles(np.zeros((max(n_pin, 1), d)))
    s.init(W)
    s.set_state(W, np.zeros((m, d, d)), np.zeros((m, d, d)), np.zeros((m, d, d)))
    s.energy(W)
    s.energy()
    g = np.zeros((n, d))
    assert s.gradient(W, out=g) is g
    out = np.zeros((n, d))
    assert s.W(out) is out and lib.calls[-1][1][1].value == out.ctypes.data
    assert s.penalties().shape == (m,)
    db = np.zeros((max(n_pin, 1), d))
    assert s.backward_unrolled(W, out=db) is db
    names = [c[0] for c in lib.calls]
    assert names == ["ffa_set_handles", "ffa_init", "ffa_set_state", "ffa_energy", "ffa_energy", "ffa_gradient",
                     "ffa_get_W", "ffa_get_penalties", "ffa_backward_unrolled"]
    torch = pytest.importorskip("torch")
    Wt = torch.zeros(n, d, dtype=torch.float64)
    s.init(Wt)
    assert s.W(Wt) is Wt and lib.calls[-1][1][1].value == Wt.data_ptr()
    b = object.__new__(S.BatchSolver)
    blib = _RecordingLib()
    b._lib, b._b, b.k, b.n, b.d = blib, None, 2, [n, n + 2], [d, 3]
    b.init([np.zeros((n, d)), torch.zeros(n + 2, 3, dtype=torch.float64)])
    o = np.zeros((n + 2, 3))
    assert b.W(1, out=o) is o and [c[0] for c in blib.calls] == ["ffa_batch_init", "ffa_batch_get_W"]


def test_constructors_pass_valid_workloads_to_the_library():
    """On a machine without a GPU, valid workloads get through the binding's checks
    and fail inside the library with FFA_ERR_CUDA (no CPU fallback), not with a
    refusal by the binding."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300._native import STATUS_NAMES, FFAError
    disk = wk.uv_disk(grid=6, seed=3)
    surf = wk.uv_heightfield(grid=6, seed=4)
    cube = wk.cube_deform(cells=2, seed=5)
    for wl in (disk, surf, cube):
        with pytest.raises(FFAError) as e:
            S.Solver.from_workload(wl)
        assert STATUS_NAMES[e.value.status] == "FFA_ERR_CUDA"
    with pytest.raises(FFAError) as e:
        S.Solver(disk.V, disk.T)                  # no pins: vertex 0 is held by the library
    assert STATUS_NAMES[e.value.status] == "FFA_ERR_CUDA"
    with pytest.raises(FFAError) as e:
        S.tutte(disk.V, disk.T, disk.pins, disk.pin_pos)
    assert STATUS_NAMES[e.value.status] == "FFA_ERR_CUDA"
    with pytest.raises(FFAError) as e:
        S.BatchSolver(wk.batched_meshes(count=2, m_min=200, m_max=400) + [cube])
    assert STATUS_NAMES[e.value.status] == "FFA_ERR_CUDA"


def test_cuda_tensors_are_synchronized_before_the_library_reads_them(monkeypatch):
    """The branch a CUDA tensor takes, run on the CPU: the tensor class is made to
    report itself as a CUDA tensor and the device synchronization is recorded.
    Inputs (converted or not) and outputs are synchronized on their own device
    before their pointer is returned; host tensors are not."""
    torch = pytest.importorskip("torch")
    seen = []
    monkeypatch.setattr(torch.cuda, "synchronize", lambda device=None: seen.append(device))
    S._ptr(torch.zeros(4, dtype=torch.float64), np.float64, 4, "W")
    S._out(torch.zeros(4, dtype=torch.float64), 4, "out")
    assert seen == []
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True))
    a = torch.zeros(4, dtype=torch.float64)
    p, keep = S._ptr(a, np.float64, 4, "W")
    assert keep is a and seen == [a.device]
    S._ptr(torch.zeros(4, dtype=torch.float32), np.float64, 4, "W")
    S._out(a, 4, "out")
    assert seen == [a.device] * 3
