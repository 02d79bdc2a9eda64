"""Pins of the oracle's anisotropic scattering (Eqs. (3)-(8)): the harmonics against
Legendre polynomials and the quadrature, the moment iteration against the
isotropic oracle and an infinite-medium solution.  The dense brute-force pin of the
moment form is in test_oracle_bruteforce.py."""
import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle
from oracle import harmonics
from paper_1906_04017_gb300 import workloads as W


@pytest.mark.parametrize("order, L", [(4, 1), (8, 3), (12, 4)])
def test_harmonics_are_orthonormal_under_the_quadrature(order, L):
    """sum_d w_d Yh_k Yh_k' = 4 pi delta_kk' (LQ_N integrates these products exactly)."""
    om, w = oracle.lqn(order)
    Y = harmonics.yhat(om, L)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - 4 * np.pi * np.eye(Y.shape[1])).max() < 1e-12


def test_addition_theorem():
    """Eq. (4): sum_m Yh_nm(a) Yh_nm(b) = (2n + 1) P_n(a . b) on random directions."""
    rng = np.random.default_rng(0)
    a = rng.normal(size=(50, 3)); a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = rng.normal(size=(50, 3)); b /= np.linalg.norm(b, axis=1, keepdims=True)
    L = 5
    Ya, Yb = harmonics.yhat(a, L), harmonics.yhat(b, L)
    mu = np.sum(a * b, axis=1)
    for n in range(L + 1):
        ks = slice(n * n, (n + 1) * (n + 1))
        lhs = np.sum(Ya[:, ks] * Yb[:, ks], axis=1)
        assert np.allclose(lhs, (2 * n + 1) * eval_legendre(n, mu), atol=1e-12)


def test_order_zero_is_the_isotropic_oracle():
    wl = W.random_small(3, 2, 2, order=4, G=2, seed=3, psi_inc=True)
    P = oracle.OracleProblem(wl)
    iso = P.source_iterate(1e-14, 500)
    mom = P.source_iterate_moments(np.zeros((1, 2, 12)), 1e-14, 500)
    assert iso["iters"] == mom["iters"]
    assert np.allclose(mom["phi"][:, :, 0], iso["phi"], rtol=1e-13, atol=0)


def test_vanishing_higher_moments_leave_the_scalar_flux_unchanged():
    """sigma_{s,n} = 0 for n >= 1: the scalar flux is the isotropic one while the
    higher flux moments (the angular shape of psi) are tallied."""
    wl = W.random_small(2, 3, 2, order=6, G=1, seed=4, psi_inc=True)
    P = oracle.OracleProblem(wl)
    iso = P.source_iterate(1e-14, 500)
    mom = P.source_iterate_moments(np.zeros((3, 1, 12)), 1e-14, 500)
    assert np.allclose(mom["phi"][:, :, 0], iso["phi"], rtol=1e-12, atol=0)
    assert np.abs(mom["phi"][:, :, 1:]).max() > 1e-3 * np.abs(iso["phi"]).max()


def test_infinite_medium_constant_solution_with_anisotropic_scattering():
    """Inflow psi = Q / (4 pi sigma_a) on every face: an isotropic psi has no moments
    above 0 (orthogonality under the quadrature), so anisotropic scattering leaves the
    constant solution phi = Q / sigma_a in every cell and node."""
    n = 3
    wl = W.random_small(n, n, n, order=6, G=1, seed=5)
    sigt, sigs, q = 2.0, 1.5, 0.7
    wl["sigt"][:] = sigt
    wl["sigs"][:] = sigs
    wl["q"][:] = q
    wl["psi_inc"][:] = q / (4 * np.pi * (sigt - sigs))
    sigs_n = np.stack([wl["sigs"], 0.6 * wl["sigs"], 0.2 * wl["sigs"]])
    r = oracle.OracleProblem(wl).source_iterate_moments(sigs_n, 1e-14, 2000)
    assert np.allclose(r["phi"][:, :, 0], q / (sigt - sigs), rtol=1e-10, atol=0)
    assert np.abs(r["phi"][:, :, 1:]).max() < 1e-10 * q / (sigt - sigs)


def test_forward_peaked_scattering_carries_flux_further():
    """A physical sanity check of the sign convention: with the same total scattering,
    forward-peaked scattering (sigma_{s,1} > 0) lets more particles cross a slab-like
    box than backward-peaked scattering does."""
    wl = W.random_small(6, 2, 2, order=6, G=1, seed=6, lengths=(6.0, 1.0, 1.0))
    wl["sigt"][:] = 1.0
    wl["sigs"][:] = 0.9
    wl["q"][:] = 0.0
    wl["psi_inc"][:] = 0.0
    wl["psi_inc"][0, 0] = 1.0          # inflow on x = 0 only
    P = oracle.OracleProblem(wl)
    far = []
    for g1 in (0.7, -0.7):
        sigs_n = np.stack([wl["sigs"], g1 * wl["sigs"]])
        r = P.source_iterate_moments(sigs_n, 1e-12, 2000)
        far.append(r["phi"][0, 5::6, 0].sum())     # the cells at the far end x = 5
    assert far[0] > 1.2 * far[1]
