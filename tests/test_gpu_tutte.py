"""The Tutte initializer on the GPU (ffa_tutte) against the oracle (oracle/tutte.py)."""
import numpy as np
import pytest

from oracle import tutte as ot
from paper_2107_05200_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("grid", [6, 48, 200])
def test_disk_matches_the_oracle_and_is_flip_free(grid):
    _need_gpu()
    from paper_2107_05200_gb300.solver import tutte
    wl = wk.uv_disk(grid=grid, seed=41, target_flip=None, sigma=0.0)
    W, rel = tutte(wl.V, wl.T, wl.pins, wl.pin_pos)
    Wo = ot.tutte(wl.V, wl.T, wl.pins, wl.pin_pos)
    assert rel < 1e-12
    assert np.abs(W - Wo).max() < 1e-10
    np.testing.assert_array_equal(W[wl.pins], wl.pin_pos)
    assert wk.flipped_fraction(W, wl.T) == 0.0


def test_surface_and_volume_match_the_oracle():
    _need_gpu()
    from paper_2107_05200_gb300.solver import tutte
    # heightfield surface (d_in = 3, d = 2): its grid boundary to the unit circle
    wl = wk.uv_heightfield(grid=24, seed=42)
    n = int(round(np.sqrt(wl.n)))
    ring = np.r_[np.arange(n), np.arange(2 * n - 1, n * n, n), np.arange(n * n - 2, n * n - n - 1, -1),
                 np.arange(n * (n - 2), 0, -n)]
    t = np.linspace(0, 2 * np.pi, len(ring), endpoint=False)
    circ = np.stack([np.cos(t), -np.sin(t)], 1)
    W, rel = tutte(wl.V, wl.T, ring, circ)
    Wo = ot.tutte(wl.V, wl.T, ring, circ)
    assert rel < 1e-12 and np.abs(W - Wo).max() < 1e-10
    # cube volume: the bottom face and the top handles held (3D Tutte can flip tets)
    cube = wk.cube_deform(cells=12, seed=43)
    W3, rel3 = tutte(cube.V, cube.T, cube.pins, cube.pin_pos)
    W3o = ot.tutte(cube.V, cube.T, cube.pins, cube.pin_pos)
    assert rel3 < 1e-12 and np.abs(W3 - W3o).max() / np.abs(W3o).max() < 1e-10


def test_invalid_inputs():
    _need_gpu()
    from paper_2107_05200_gb300._native import FFAError
    from paper_2107_05200_gb300.solver import tutte
    wl = wk.uv_disk(grid=6, seed=44, target_flip=None, sigma=0.0)
    with pytest.raises(FFAError):
        tutte(wl.V, wl.T, np.r_[wl.pins, wl.pins[:1]], np.r_[wl.pin_pos, wl.pin_pos[:1]])
    with pytest.raises(FFAError):
        tutte(wl.V, wl.T, np.array([wl.n + 5]), np.zeros((1, 2)))
