"""The volume-correspondence workload (Sec. Results, "Volume Correspondence") on
the oracle: the boundary of the first volume held on the second surface, the
interior started from the minimizer of Tutte's energy (App. A), which folds some
tetrahedra, and the method reaching its termination test (eq.
primaldualthresholds) with no flipped tetrahedron, as the paper reports for this
application."""
import numpy as np

from oracle import admm
from paper_2107_05200_gb300 import workloads as wk


def test_boundary_is_held_on_the_second_surface():
    wl = wk.volume_correspondence(cells=6)
    h = 1.0 / 6
    on_face = np.any((wl.V < 0.5 * h) | (wl.V > 1 - 0.5 * h), axis=1)
    assert set(wl.pins.tolist()) == set(np.nonzero(on_face)[0].tolist())
    np.testing.assert_allclose(wl.pin_pos, wk.twist_bend_map(wl.V[wl.pins]), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(wl.W0[wl.pins], wl.pin_pos)
    # the map restricted to the boundary is the analytic twist and bend: a rigid
    # motion of the bottom face (z = 0: no twist, bend angle 0) is the identity
    bottom = wl.pins[wl.V[wl.pins, 2] < 0.5 * h]
    np.testing.assert_allclose(wk.twist_bend_map(wl.V[bottom]), wl.V[bottom], atol=1e-15)


def test_tutte_start_folds_and_the_method_ends_flip_free():
    wl = wk.volume_correspondence(cells=6)
    assert wl.meta["flipped0"] > 0.0
    o = admm.Oracle.from_workload(wl)
    s, st = o.run(wl.W0, 200, stop_at_tol=True)
    assert st.e_prim <= st.thr_prim and st.e_dual <= st.thr_dual, (st.k, st.e_prim, st.thr_prim)
    assert wk.flipped_fraction(s.W, wl.T) == 0.0
    assert st.k < 200


def test_a_boundary_map_that_inverts_a_pinned_tet_is_refused():
    import pytest
    with pytest.raises(ValueError):
        wk.volume_correspondence(cells=2, twist=9.0, radius=0.6)
