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


def test_blocked_64_follows_its_recipe():
    """64^3 cells on a 10^3 box, LQ_8, 8 groups; sigma_t constant on each 8^3 block and
    lognormal(0, 1) over the blocks; scattering ratio U[0.3, 0.9] per block, the same in
    every group; downscatter-only transfer; q = 1 in group 0 on one 16^3 box only."""
    wl = W.blocked_64()
    assert (wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["order"]) == (64, 64, 64, 10.0, 8)
    G = wl["sigt"].shape[0]
    assert G == 8
    sig = wl["sigt"].reshape(G, 8, 8, 8, 8, 8, 8)      # [g][bk][k][bj][j][bi][i]
    blocks = sig[:, :, 0, :, 0, :, 0]
    assert np.all(sig == blocks[:, :, None, :, None, :, None])
    logs = np.log(blocks).ravel()                        # 8 groups x 512 blocks
    assert abs(logs.mean()) < 0.1 and abs(logs.std() - 1.0) < 0.05
    ratio = wl["sigs"] / wl["sigt"]
    assert np.allclose(ratio, ratio[0][None, :]) and ratio.min() >= 0.3 and ratio.max() <= 0.9
    x = wl["xfer"]
    # row g' holds where group g' scatters to: only g >= g' (downscatter), all of it
    assert np.all(x[np.tril_indices(G, -1)] == 0.0) and np.allclose(x.sum(axis=1), 1.0)
    src = wl["q"][0].reshape(64, 64, 64) > 0
    assert src.sum() == 16 ** 3 and np.all(wl["q"][1:] == 0.0) and np.all(wl["q"][0][wl["q"][0] > 0] == 1.0)
    k, j, i = np.nonzero(src)
    assert (i.max() - i.min(), j.max() - j.min(), k.max() - k.min()) == (15, 15, 15)


def test_spheres_96_background_and_sources():
    """Background sigma_t = 0.1 with scattering ratio 0.5; sources (q = 1, group 0 only)
    lie inside spheres, never in the background."""
    wl = W.spheres_96()
    assert (wl["nx"], wl["order"], wl["sigt"].shape[0]) == (96, 12, 16)
    bg = np.all(wl["sigt"] == 0.1, axis=0)
    assert bg.mean() > 0.2
    assert np.allclose(wl["sigs"][:, bg], 0.05)
    src = wl["q"][0] > 0
    assert src.any() and not np.any(src & bg) and np.all(wl["q"][1:] == 0.0)


def test_onecell_problems_follow_the_training_distribution():
    """Directions on the unit sphere, cell sizes in [0.1, 1], sigma_t lognormal(0, 1.5),
    sources and upwind values in [0, 1]."""
    x = W.onecell_problems(20000, seed=9)
    assert np.allclose(np.linalg.norm(x[:, 0:3], axis=1), 1.0)
    assert np.all(np.abs(np.sign(x[:, 0:3]).mean(axis=0)) < 0.05)
    assert x[:, 3:6].min() >= 0.1 and x[:, 3:6].max() <= 1.0
    ls = np.log(x[:, 6])
    assert abs(ls.mean()) < 0.05 and abs(ls.std() - 1.5) < 0.05
    assert x[:, 7:27].min() >= 0.0 and x[:, 7:27].max() <= 1.0
