"""GPU parity of anisotropic scattering (Eqs. (3)-(8)) against the FP64 oracle's moment
sweep and moment source iteration, through the C ABI.  The library holds moments in
the layout [G][K][ncell][8], the oracle in [G][ncell][K][8]."""
import numpy as np
import pytest
import torch

import oracle
from paper_1906_04017_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def cuda(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def legendre_moments(wl, L, seed):
    """sigma_{s,n} = g^n sigma_s with a per-cell anisotropy g in [-0.6, 0.8]: [L+1, G, C]."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(-0.6, 0.8, size=wl["sigs"].shape)
    return np.stack([wl["sigs"] * g ** n for n in range(L + 1)])


def to_oracle(m):     # [G, K, C, 8] -> [G, C, K, 8]
    return np.ascontiguousarray(np.transpose(m, (0, 2, 1, 3)))


def moment_err(got, ref):
    """max over (group, moment) of max |got - ref| / max |ref of moment 0 in that group|
    (arrays in the oracle layout [G, C, K, 8])."""
    worst = 0.0
    for g in range(ref.shape[0]):
        scale = np.abs(ref[g, :, 0]).max()
        worst = max(worst, float(np.abs(got[g] - ref[g]).max() / scale))
    return worst


@pytest.mark.parametrize("order, L", [(2, 1), (4, 2), (8, 3), (12, 1), (8, 1)])
def test_moment_sweep_matches_oracle(sn, order, L):
    wl = W.random_small(3, 4, 2, order=order, G=2, seed=40 + L, psi_inc=True)
    sig_n = legendre_moments(wl, L, seed=order)
    P = sn.Problem(wl)
    P.set_scattering_order(L, sig_n[1:])
    K = (L + 1) ** 2
    rng = np.random.default_rng(order + L)
    S = rng.uniform(-0.3, 1.0, (P.G, K, P.ncell, 8)).astype(np.float32)
    S[:, 0] = np.abs(S[:, 0])
    phi = P.sweep(cuda(S)).cpu().numpy()
    bal = P.balance()
    P.close()
    ref, tal = oracle.OracleProblem(wl).sweep_moments(to_oracle(S.astype(np.float64)), sig_n)
    assert moment_err(to_oracle(phi), ref) < 1e-5
    # particle balance of the sweep (moments above 0 integrate to zero over directions)
    assert abs(bal[0] + bal[1] - bal[2] - bal[3]) < 1e-5 * (bal[2] + bal[3])
    assert np.allclose(bal[:3], tal[:3], rtol=1e-5)


@pytest.mark.parametrize("use_graph", [True, False])
def test_moment_source_iteration_matches_oracle(sn, use_graph):
    """Four source iterations from zero (moment source, sweep, octant reduction)."""
    wl = W.random_small(4, 3, 3, order=4, G=2, seed=50, psi_inc=True)
    L = 2
    sig_n = legendre_moments(wl, L, seed=51)
    P = sn.Problem(wl)
    P.set_scattering_order(L, sig_n[1:])
    r = P.source_iterate(tol=0.0, max_it=4, use_graph=use_graph, allow_noconv=True)
    phi = r["phi"].cpu().numpy()
    P.close()
    ref = oracle.OracleProblem(wl).source_iterate_moments(sig_n, 0.0, 4)
    assert r["iters"] == ref["iters"] == 4
    assert moment_err(to_oracle(phi), ref["phi"]) < 1e-5
    assert r["change_max"] == pytest.approx(ref["change_max"], rel=1e-4)


def test_converged_fp64_matches_oracle(sn):
    wl = W.random_small(3, 3, 2, order=6, G=2, seed=52, psi_inc=True)
    L = 3
    sig_n = legendre_moments(wl, L, seed=53)
    P = sn.Problem(wl, fp64=True)
    P.set_scattering_order(L, sig_n[1:])
    r = P.source_iterate(tol=1e-13, max_it=2000)
    phi = r["phi"].cpu().numpy()
    P.close()
    ref = oracle.OracleProblem(wl).source_iterate_moments(sig_n, 1e-14, 3000)
    assert r["converged"] and ref["converged"]
    assert moment_err(to_oracle(phi), ref["phi"]) < 1e-11


def test_converged_fp32_matches_oracle(sn):
    wl = W.random_small(4, 4, 3, order=8, G=2, seed=54, psi_inc=True)
    L = 1
    sig_n = legendre_moments(wl, L, seed=55)
    P = sn.Problem(wl)
    P.set_scattering_order(L, sig_n[1:])
    r = P.source_iterate(tol=1e-6, max_it=500)
    phi = r["phi"].cpu().numpy()
    P.close()
    ref = oracle.OracleProblem(wl).source_iterate_moments(sig_n, 1e-14, 3000)
    assert moment_err(to_oracle(phi), ref["phi"]) < 2e-5


def test_order_zero_restores_the_isotropic_sweep(sn):
    wl = W.random_small(3, 2, 4, order=8, G=2, seed=56, psi_inc=True)
    S = cuda(np.random.default_rng(3).uniform(0, 1, (2, 24, 8)))
    P = sn.Problem(wl)
    iso = P.sweep(S).cpu().numpy()
    P.set_scattering_order(1, legendre_moments(wl, 1, 57)[1:])
    P.set_scattering_order(0)
    back = P.sweep(S).cpu().numpy()
    P.close()
    assert np.array_equal(iso, back)


def test_other_modes_are_rejected(sn):
    wl = W.random_small(2, 2, 2, order=4, G=1, seed=58)
    P = sn.Problem(wl)
    P.set_scattering_order(1, legendre_moments(wl, 1, 59)[1:])
    P.surrogate_init(0)
    S = P.flux_tensor()
    try:
        for mode in (sn.ANN, sn.ANN_GATED):
            with pytest.raises(sn.SnError) as e:
                P.sweep(S, mode=mode)
            assert e.value.status == sn.SN_EINVAL
        with pytest.raises(sn.SnError):
            P.set_scattering_order(4, np.zeros((4, 1, 8)))
    finally:
        P.close()


def test_moment_sweep_full_size_sampled_group(sn):
    """blocked_64 (64^3, LQ_8, 8 groups) with linearly anisotropic scattering, in the
    launch configuration of the measurements: one sweep of every group from random
    source moments, the last group recomputed by the oracle."""
    wl = W.blocked_64()
    L = 1
    sig_n = legendre_moments(wl, L, seed=60)
    P = sn.Problem(wl)
    P.set_scattering_order(L, sig_n[1:])
    K = 4
    rng = np.random.default_rng(61)
    S = rng.uniform(-0.2, 1.0, (P.G, K, P.ncell, 8)).astype(np.float32)
    S[:, 0] = np.abs(S[:, 0])
    phi = P.sweep(cuda(S)).cpu().numpy()
    P.close()
    g = P.G - 1
    ref, _ = oracle.OracleProblem(wl).sweep_moments(to_oracle(S.astype(np.float64)), sig_n, groups=(g, g + 1))
    assert moment_err(to_oracle(phi)[g:g + 1], ref[g:g + 1]) < 1e-5
