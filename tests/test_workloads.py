"""Host-side checks of the synthetic input generators (no method arithmetic)."""
import numpy as np

from paper_1906_04017_gb300 import workloads as W


def test_deformed_vertices_keep_the_box():
    wl = W.random_small(4, 3, 5, order=4, G=1, seed=1)
    box = W.box_vertices(wl)
    v = W.deformed_vertices(wl, 0.2, seed=3)
    assert v.shape == ((4 + 1) * (3 + 1) * (5 + 1), 3)
    lo, hi = box.min(axis=0), box.max(axis=0)
    for a in range(3):
        on = np.isclose(box[:, a], lo[a]) | np.isclose(box[:, a], hi[a])
        assert np.array_equal(v[on, a], box[on, a])          # boundary planes kept
        assert np.any(v[~on, a] != box[~on, a])               # interior moved
    h = (hi - lo) / np.array([4, 3, 5])
    assert np.all(np.abs(v - box) <= 0.2 * h + 1e-15)


def test_box_vertex_order():
    wl = W.random_small(2, 3, 4, order=4, G=1, seed=2, lengths=(2.0, 3.0, 4.0))
    v = W.box_vertices(wl)
    idx = lambda i, j, k: i + 3 * (j + 4 * k)
    assert np.allclose(v[idx(1, 2, 3)], [1.0, 2.0, 3.0])
    assert np.allclose(v[idx(2, 0, 0)], [2.0, 0.0, 0.0])


def test_octant_problems_lie_in_their_octants():
    m = 50
    x = W.octant_problems(m, seed=4)
    lo, hi = W.octant_net_ranges()
    for o in range(8):
        rows = x[o * m:(o + 1) * m]
        for a in range(3):
            s = -1.0 if (o >> a) & 1 else 1.0
            assert np.all(s * rows[:, a] > 0)
        assert np.allclose(np.linalg.norm(rows[:, 0:3], axis=1), 1.0)
        for j, col in ((12, 0), (13, 1)):
            assert np.all(rows[:, col] >= lo[o, j]) and np.all(rows[:, col] <= hi[o, j])
