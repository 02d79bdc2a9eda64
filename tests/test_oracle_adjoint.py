"""Pins of the oracle's discrete adjoint (gradients of a detector response with
respect to sigma_t, sigma_s and q; not in the paper, defined by the discrete
system of Sec. 2): central finite differences of the FP64 forward solve, the
exact linearity of the response in q, and a dense transposed solve of the whole
discrete system on a 2x2x2 mesh."""
import numpy as np
import pytest

import oracle
from paper_1906_04017_gb300 import workloads as W
from test_oracle_bruteforce import kron_elements


def corner_response(wl, n=2):
    """dR/dphi of R = sum_g integral of phi_g over the n^3 corner cells."""
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    G = wl["sigt"].shape[0]
    vol = wl["lx"] / nx * wl["ly"] / ny * wl["lz"] / nz
    r = np.zeros((G, nx * ny * nz, 8))
    i, j, k = W.cell_ijk(wl)
    r[:, (i < n) & (j < n) & (k < n), :] = vol / 8.0
    return r


def response(wl, r):
    P = oracle.OracleProblem(wl)
    phi = P.source_iterate(1e-15, 5000)["phi"]
    return float(np.sum(r * phi)), phi


@pytest.fixture(scope="module")
def case():
    wl = W.random_small(4, 3, 3, order=4, G=2, seed=17, psi_inc=True)
    wl["sigs"] = 0.6 * wl["sigt"]
    r = corner_response(wl)
    R, phi = response(wl, r)
    adj = oracle.OracleProblem(wl).adjoint(phi, r)
    return wl, r, R, phi, adj


@pytest.mark.parametrize("field,key", [("sigt", "grad_sigt"), ("sigs", "grad_sigs"), ("q", "grad_q")])
def test_gradient_matches_central_differences(case, field, key):
    wl, r, R, phi, adj = case
    assert adj["converged"]
    rng = np.random.default_rng(3)
    G, n = wl["sigt"].shape
    picks = [(g, c) for g in range(G) for c in rng.choice(n, 4, replace=False)]
    for g, c in picks:
        base = wl[field][g, c]
        h = 1e-5 * max(abs(base), 1e-2)
        vals = []
        for sgn in (1, -1):
            w2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in wl.items()}
            w2[field][g, c] = base + sgn * h
            if field == "sigt":      # keep sigma_s fixed while sigma_t moves
                w2["sigs"] = wl["sigs"].copy()
            vals.append(response(w2, r)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        got = adj[key][g, c]
        assert abs(got - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(R)), (field, g, c, got, fd)


def test_response_is_linear_in_q():
    """With vacuum inflow R is linear and homogeneous in q, so R = sum dR/dq * q."""
    wl = W.random_small(3, 4, 2, order=6, G=3, seed=4)
    wl["q"] = np.random.default_rng(1).uniform(0.1, 1.0, wl["q"].shape)
    r = corner_response(wl, 1)
    R, phi = response(wl, r)
    adj = oracle.OracleProblem(wl).adjoint(phi, r)
    assert abs(np.sum(adj["grad_q"] * wl["q"]) - R) < 1e-12 * abs(R)


def test_adjoint_matches_dense_transposed_solve():
    """On a 2x2x2 mesh the whole system (every direction, group, cell and node,
    upwind couplings, scattering) is one dense matrix A_tot; the adjoint scalar flux
    is sum_d of lambda = A_tot^{-T} Phi^T r."""
    wl = W.random_small(2, 2, 2, order=4, G=2, seed=23, psi_inc=True)
    wl["sigs"] = 0.7 * wl["sigt"]
    nx, ny, nz = 2, 2, 2
    h = (wl["lx"] / nx, wl["ly"] / ny, wl["lz"] / nz)
    om, w = oracle.lqn(4)
    G, nc, nd = 2, 8, len(w)
    M, Gm, F = kron_elements(h)
    pos = {}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = i + nx * (j + ny * k)
                for n in range(8):
                    pos[(c, n)] = (i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1))
    N = nd * G * nc * 8
    idx = lambda d, g, c, n: ((d * G + g) * nc + c) * 8 + n
    A = np.zeros((N, N))
    for d in range(nd):
        o = om[d]
        for g in range(G):
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        c = i + nx * (j + ny * k)
                        loc = sum(o[a] * Gm[a] for a in range(3)) + wl["sigt"][g, c] * M
                        for a in range(3):
                            side = 0 if o[a] > 0 else 1
                            Ff = F[(a, side)]
                            loc = loc + abs(o[a]) * Ff
                            ijk = [i, j, k]
                            ijk[a] += -1 if side == 0 else 1
                            if 0 <= ijk[a] < 2:
                                cu = ijk[0] + nx * (ijk[1] + ny * ijk[2])
                                for jn in range(8):
                                    if not np.any(Ff[:, jn]):
                                        continue
                                    ju = [m for m in range(8) if pos[(cu, m)] == pos[(c, jn)]][0]
                                    for kn in range(8):
                                        A[idx(d, g, c, kn), idx(d, g, cu, ju)] -= abs(o[a]) * Ff[kn, jn]
                        for kn in range(8):
                            for jn in range(8):
                                A[idx(d, g, c, kn), idx(d, g, c, jn)] += loc[kn, jn]
                        for gp in range(G):
                            coef = wl["xfer"][gp, g] * wl["sigs"][gp, c] / (4 * np.pi)
                            for dp in range(nd):
                                for kn in range(8):
                                    for jn in range(8):
                                        A[idx(d, g, c, kn), idx(dp, gp, c, jn)] -= coef * w[dp] * M[kn, jn]
    r = corner_response(wl, 1)
    rhs = np.zeros(N)
    for d in range(nd):
        for g in range(G):
            for c in range(nc):
                rhs[idx(d, g, c, 0):idx(d, g, c, 0) + 8] = w[d] * r[g, c]
    lam = np.linalg.solve(A.T, rhs).reshape(nd, G, nc, 8)
    Lam_ref = lam.sum(axis=0)
    P = oracle.OracleProblem(wl)
    phi = P.source_iterate(1e-15, 5000)["phi"]
    adj = P.adjoint(phi, r, tol=1e-15, maxit=5000)
    assert np.allclose(adj["Lam"], Lam_ref, rtol=1e-10, atol=1e-13 * np.abs(Lam_ref).max())
