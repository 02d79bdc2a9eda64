"""Brute-force pin of the oracle's sweep + source iteration (Sec. 2, Eqs. (12)-(14)
and the scattering source iteration described after Eq. (7)).

On a 2x2x2 mesh the whole discrete problem -- every direction, group, cell and
node, with the upwind couplings between cells and the group-to-group scattering
written as explicit matrix entries -- fits in one dense matrix.  Solving it
directly gives the fixed point that source iteration must converge to.  The
element matrices here come from 1D Kronecker factors of the classic upwind
(inflow) form, and the upwind coupling is found by matching node coordinates, so
none of the oracle's assembly or gather code is reused."""
import numpy as np
import pytest

import oracle
from paper_1906_04017_gb300 import workloads as W


def kron_elements(h):
    m = lambda hh: hh / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    g = np.array([[-0.5, 0.5], [-0.5, 0.5]])          # int b_k b_j'
    e = [np.array([[1.0, 0.0], [0.0, 0.0]]), np.array([[0.0, 0.0], [0.0, 1.0]])]
    K = lambda cz, cy, cx: np.kron(cz, np.kron(cy, cx))
    mx, my, mz = m(h[0]), m(h[1]), m(h[2])
    M = K(mz, my, mx)
    G = [K(mz, my, g), K(mz, g, mx), K(g, my, mx)]
    F = {(0, 0): K(mz, my, e[0]), (0, 1): K(mz, my, e[1]),
         (1, 0): K(mz, e[0], mx), (1, 1): K(mz, e[1], mx),
         (2, 0): K(e[0], my, mx), (2, 1): K(e[1], my, mx)}
    return M, G, F


def brute_force_phi(wl):
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    h = (wl["lx"] / nx, wl["ly"] / ny, wl["lz"] / nz)
    om, w = oracle.lqn(wl["order"])
    G_ = wl["sigt"].shape[0]
    nc = nx * ny * nz
    M, Gm, F = kron_elements(h)
    pos = {}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = i + nx * (j + ny * k)
                for n in range(8):
                    key = (i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1))
                    pos[(c, n)] = key
    nd = len(w)
    N = nd * G_ * nc * 8
    idx = lambda d, g, c, n: ((d * G_ + g) * nc + c) * 8 + n
    A = np.zeros((N, N))
    rhs = np.zeros(N)
    for d in range(nd):
        o = om[d]
        for g in range(G_):
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        c = i + nx * (j + ny * k)
                        loc = sum(o[a] * Gm[a] for a in range(3)) + wl["sigt"][g, c] * M
                        src_rhs = M @ np.full(8, wl["q"][g, c] / (4 * np.pi))
                        for a in range(3):
                            side = 0 if o[a] > 0 else 1           # inflow face
                            Ff = F[(a, side)]
                            loc = loc + abs(o[a]) * Ff
                            ijk = [i, j, k]
                            ijk[a] += -1 if side == 0 else 1
                            if 0 <= ijk[a] < [nx, ny, nz][a]:
                                cu = ijk[0] + nx * (ijk[1] + ny * ijk[2])
                                for jn in range(8):
                                    if not np.any(Ff[:, jn]):
                                        continue
                                    target = pos[(c, jn)]
                                    ju = [m for m in range(8) if pos[(cu, m)] == target][0]
                                    for kn in range(8):
                                        A[idx(d, g, c, kn), idx(d, g, cu, ju)] -= abs(o[a]) * Ff[kn, jn]
                            else:
                                face = 2 * a + side
                                src_rhs = src_rhs + abs(o[a]) * Ff @ np.full(8, wl["psi_inc"][g, face])
                        for kn in range(8):
                            for jn in range(8):
                                A[idx(d, g, c, kn), idx(d, g, c, jn)] += loc[kn, jn]
                            rhs[idx(d, g, c, kn)] = src_rhs[kn]
                        # scattering: -(1/4pi) M sum_g' xfer[g'][g] sigs[g'] sum_d' w_d' psi
                        for gp in range(G_):
                            coef = wl["xfer"][gp, g] * wl["sigs"][gp, c] / (4 * np.pi)
                            if coef == 0.0:
                                continue
                            for dp in range(nd):
                                for kn in range(8):
                                    for jn in range(8):
                                        A[idx(d, g, c, kn), idx(dp, gp, c, jn)] -= coef * w[dp] * M[kn, jn]
    psi = np.linalg.solve(A, rhs).reshape(nd, G_, nc, 8)
    return np.einsum("d,dgcn->gcn", w, psi)


@pytest.mark.parametrize("G", [1, 2])
def test_bruteforce_2x2x2(G):
    wl = W.random_small(2, 2, 2, order=4, G=G, seed=21 + G, psi_inc=True)
    wl["sigs"] = 0.8 * wl["sigt"]
    phi_ref = brute_force_phi(wl)
    P = oracle.OracleProblem(wl)
    r = P.source_iterate(1e-15, 2000)
    assert np.allclose(r["phi"], phi_ref, rtol=1e-11, atol=1e-13 * np.abs(phi_ref).max())
