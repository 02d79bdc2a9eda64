"""Brute-force pin of the oracle's sweep + source iteration (Sec. 2, Eqs. (12)-(14)
and the scattering source iteration described after Eq. (7)).

On a 2x2x2 mesh the whole discrete problem -- every direction, group, cell and
node, with the upwind couplings between cells and the group-to-group scattering
written as explicit matrix entries (isotropic, or anisotropic from the Legendre
expansion of Eq. (3)) -- fits in one dense matrix.  Solving it
directly gives the fixed point that source iteration must converge to.  The
element matrices here come from 1D Kronecker factors of the classic upwind
(inflow) form, and the upwind coupling is found by matching node coordinates, so
none of the oracle's assembly or gather code is reused."""
import numpy as np
import pytest
from scipy.special import eval_legendre

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


def brute_force_psi(wl, sigs_n=None):
    """Angular flux [ndir, G, ncell, 8] of the dense solve.  sigs_n: optional Legendre
    scattering moments [L+1][G][ncell] (row 0 ignored, the workload's sigma_s); the
    scattering kernel between two directions is then written out from Eq. (3),
    sum_n (2n+1)/(4 pi) sigma_{s,n} P_n(Omega_d . Omega_d'), with Legendre
    polynomials from scipy, not from any spherical harmonic."""
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
                        # scattering: -M sum_g' xfer[g'][g] sum_d' w_d' k(d, d') psi_d' with the
                        # kernel k = sum_n (2n+1)/(4 pi) sigma_{s,n,g'} P_n(Omega_d . Omega_d')
                        for gp in range(G_):
                            if wl["xfer"][gp, g] == 0.0:
                                continue
                            for dp in range(nd):
                                kern = wl["sigs"][gp, c] / (4 * np.pi)
                                if sigs_n is not None:
                                    mu0 = float(np.dot(om[d], om[dp]))
                                    for n in range(1, len(sigs_n)):
                                        kern += (2 * n + 1) / (4 * np.pi) * sigs_n[n][gp, c] * eval_legendre(n, mu0)
                                coef = wl["xfer"][gp, g] * kern * w[dp]
                                if coef == 0.0:
                                    continue
                                for kn in range(8):
                                    for jn in range(8):
                                        A[idx(d, g, c, kn), idx(dp, gp, c, jn)] -= coef * M[kn, jn]
    psi = np.linalg.solve(A, rhs).reshape(nd, G_, nc, 8)
    return psi


def brute_force_phi(wl):
    om, w = oracle.lqn(wl["order"])
    return np.einsum("d,dgcn->gcn", w, brute_force_psi(wl))


@pytest.mark.parametrize("G", [1, 2])
def test_bruteforce_2x2x2(G):
    wl = W.random_small(2, 2, 2, order=4, G=G, seed=21 + G, psi_inc=True)
    wl["sigs"] = 0.8 * wl["sigt"]
    phi_ref = brute_force_phi(wl)
    P = oracle.OracleProblem(wl)
    r = P.source_iterate(1e-15, 2000)
    assert np.allclose(r["phi"], phi_ref, rtol=1e-11, atol=1e-13 * np.abs(phi_ref).max())


@pytest.mark.parametrize("L, G", [(1, 1), (2, 2), (3, 1)])
def test_bruteforce_anisotropic_2x2x2(L, G):
    """The moment form of the anisotropic source (Eqs. (5)-(8): flux moments and
    harmonics) converges to the dense solve whose scattering is Eq. (3) written with
    Legendre polynomials between every pair of directions."""
    from oracle import harmonics
    wl = W.random_small(2, 2, 2, order=4, G=G, seed=30 + L, psi_inc=True)
    wl["sigs"] = 0.8 * wl["sigt"]
    rng = np.random.default_rng(L)
    # Henyey-Greenstein-like moments sigma_{s,n} = g^n sigma_s, g in [-0.6, 0.8]
    gfac = rng.uniform(-0.6, 0.8, size=wl["sigs"].shape)
    sigs_n = [wl["sigs"]] + [wl["sigs"] * gfac ** n for n in range(1, L + 1)]
    psi = brute_force_psi(wl, sigs_n)
    om, w = oracle.lqn(wl["order"])
    Yh = harmonics.yhat(om, L)
    mom_ref = np.einsum("d,dk,dgcn->gckn", w, Yh, psi)
    r = oracle.OracleProblem(wl).source_iterate_moments(np.array(sigs_n), 1e-15, 3000)
    assert r["converged"]
    scale = np.abs(mom_ref[:, :, 0]).max()
    assert np.allclose(r["phi"], mom_ref, rtol=0, atol=1e-11 * scale)
