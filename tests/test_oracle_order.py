"""Pin of the property the wavefront sweep rests on: the upwind DFEM sweep's result
does not depend on the order in which cells are visited, as long as every cell comes
after its upwind neighbours (Sec. 2, the sweep after Eq. (14)).  The oracle's
lexicographic sweep is compared with a sweep that visits the hyperplanes
i' + j' + k' = s in turn, the cells of each plane in random order, with every cell
solved by the oracle's one-cell elimination: the results are identical bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1906_04017_gb300 import workloads as W


def face_node(ax, side, t):
    lo, hi = t & 1, (t >> 1) & 1
    abc = [lo, hi]
    abc.insert(ax, side)
    return abc[0] + 2 * abc[1] + 4 * abc[2]


def hyperplane_sweep(wl, d, g, S, rng):
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    h = (wl["lx"] / nx, wl["ly"] / ny, wl["lz"] / nz)
    om, _ = oracle.lqn(wl["order"])
    o = om[d]
    psi = np.full((nx * ny * nz, 8), np.nan)
    # distance of a cell from the inflow corner along each axis
    cells = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    dist = lambda c: sum(c[a] if o[a] >= 0 else (nx, ny, nz)[a] - 1 - c[a] for a in range(3))
    for s in range(nx + ny + nz - 2):
        plane = [c for c in cells if dist(c) == s]
        for q in rng.permutation(len(plane)):
            i, j, k = plane[q]
            c = i + nx * (j + ny * k)
            x = np.zeros(27)
            x[0:3], x[3:6], x[6] = o, h, wl["sigt"][g, c]
            x[7:15] = S[c]
            for a in range(3):
                fin = 0 if o[a] >= 0 else 1
                idx = [i, j, k]
                idx[a] += -1 if fin == 0 else 1
                if 0 <= idx[a] < (nx, ny, nz)[a]:
                    cu = idx[0] + nx * (idx[1] + ny * idx[2])
                    up = [psi[cu, face_node(a, 1 - fin, t)] for t in range(4)]
                    assert not np.any(np.isnan(up)), "upwind cell not yet solved"
                else:
                    up = [wl["psi_inc"][g, 2 * a + fin]] * 4
                x[15 + 4 * a:19 + 4 * a] = up
            psi[c] = oracle.cell_solve(x)[0]
    return psi


@pytest.mark.parametrize("order", [2, 4])
def test_hyperplane_order_gives_the_lexicographic_result(order):
    wl = W.random_small(4, 3, 5, order=order, G=2, seed=21, psi_inc=True)
    P = oracle.OracleProblem(wl)
    rng = np.random.default_rng(0)
    S = rng.uniform(0.0, 1.0, (P.ncell, 8))
    for d in range(P.ndir):
        for g in range(2):
            lex, _ = P.sweep_dir(d, g, S)
            hyp = hyperplane_sweep(wl, d, g, S, rng)
            assert np.array_equal(lex, hyp)
