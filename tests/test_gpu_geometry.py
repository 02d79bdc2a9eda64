"""GPU parity of the general hexahedral cells (trilinear maps, element matrices
computed on the device) against the FP64 oracle's sweep on the same vertices,
through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1906_04017_gb300 import workloads as W
from _parity import norm_err

pytestmark = pytest.mark.gpu


def cuda(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def test_box_vertices_match_the_box_cells(sn):
    wl = W.random_small(3, 4, 2, order=8, G=2, seed=70, psi_inc=True)
    S = cuda(np.random.default_rng(0).uniform(0, 1, (2, 24, 8)))
    P = sn.Problem(wl)
    box = P.sweep(S).cpu().numpy()
    P.set_geometry(W.box_vertices(wl))
    gen = P.sweep(S).cpu().numpy()
    P.set_geometry(None)
    back = P.sweep(S).cpu().numpy()
    P.close()
    assert norm_err(gen, box) < 1e-5
    assert np.array_equal(back, box)


@pytest.mark.parametrize("order", [2, 4, 8, 12])
def test_deformed_sweep_matches_oracle(sn, order):
    wl = W.random_small(3, 4, 2, order=order, G=2, seed=71, psi_inc=True)
    # LQ_8 and LQ_12 have directions within 13 and 10 degrees of a face plane: the
    # faces may tilt less before a face's inflow side changes
    xyz = W.deformed_vertices(wl, 0.06 if order <= 4 else 0.03, seed=order)
    rng = np.random.default_rng(order)
    S = rng.uniform(0.0, 1.0, (2, 24, 8)).astype(np.float32)
    P = sn.Problem(wl)
    P.set_geometry(xyz)
    phi = P.sweep(cuda(S)).cpu().numpy()
    bal = P.balance()
    P.close()
    ref, tal = oracle.OracleProblem(wl, xyz=xyz).sweep(S.astype(np.float64))
    assert norm_err(phi, ref) < 1e-5
    assert abs(bal[0] + bal[1] - bal[2] - bal[3]) < 1e-5 * (bal[2] + bal[3])
    assert np.allclose(bal, tal, rtol=1e-5)


@pytest.mark.parametrize("use_graph", [True, False])
def test_deformed_source_iteration_matches_oracle(sn, use_graph):
    wl = W.random_small(4, 3, 3, order=4, G=2, seed=72, psi_inc=True)
    xyz = W.deformed_vertices(wl, 0.08, seed=5)
    P = sn.Problem(wl)
    P.set_geometry(xyz)
    r = P.source_iterate(tol=0.0, max_it=4, use_graph=use_graph, allow_noconv=True)
    phi = r["phi"].cpu().numpy()
    P.close()
    ref = oracle.OracleProblem(wl, xyz=xyz).source_iterate(0.0, 4)
    assert norm_err(phi, ref["phi"]) < 1e-5


def test_deformed_fp64_converged_matches_oracle(sn):
    wl = W.random_small(3, 3, 3, order=6, G=2, seed=73, psi_inc=True)
    xyz = W.deformed_vertices(wl, 0.04, seed=6)
    P = sn.Problem(wl, fp64=True)
    P.set_geometry(xyz)
    r = P.source_iterate(tol=1e-13, max_it=2000)
    phi = r["phi"].cpu().numpy()
    P.close()
    ref = oracle.OracleProblem(wl, xyz=xyz).source_iterate(1e-14, 3000)
    assert r["converged"]
    assert norm_err(phi, ref["phi"]) < 1e-11


def test_too_deformed_mesh_is_rejected(sn):
    """Vertices moved by up to 45% of a cell flip some face's inflow side for LQ_12
    directions (or fold a cell): rejected, and the handle keeps its box cells."""
    wl = W.random_small(4, 4, 4, order=12, G=1, seed=74, psi_inc=True)
    S = cuda(np.random.default_rng(1).uniform(0, 1, (1, 64, 8)))
    P = sn.Problem(wl)
    before = P.sweep(S).cpu().numpy()
    with pytest.raises(sn.SnError) as e:
        P.set_geometry(W.deformed_vertices(wl, 0.45, seed=7))
    assert e.value.status == sn.SN_EINVAL
    after = P.sweep(S).cpu().numpy()
    P.close()
    assert np.array_equal(before, after)


def test_other_modes_are_rejected(sn):
    wl = W.random_small(2, 2, 2, order=4, G=1, seed=75)
    P = sn.Problem(wl)
    P.set_geometry(W.deformed_vertices(wl, 0.05, seed=8))
    P.surrogate_init(0)
    try:
        with pytest.raises(sn.SnError) as e:
            P.sweep(P.flux_tensor(), mode=sn.ANN)
        assert e.value.status == sn.SN_EINVAL
        with pytest.raises(sn.SnError):
            P.set_scattering_order(1, np.zeros((1, 1, 8)))
    finally:
        P.close()


def test_deformed_blocked_32_sampled_group(sn):
    """The 32^3, LQ_8, 4-group blocked workload on a deformed mesh (vertices moved by up
    to 3% of a cell): one sweep of every group, the last group recomputed by the oracle."""
    wl = W.blocked_32()
    xyz = W.deformed_vertices(wl, 0.03, seed=9)
    P = sn.Problem(wl)
    P.set_geometry(xyz)
    rng = np.random.default_rng(10)
    S = rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32)
    phi = P.sweep(cuda(S)).cpu().numpy()
    P.close()
    g = P.G - 1
    ref, _ = oracle.OracleProblem(wl, xyz=xyz).sweep(S.astype(np.float64), groups=(g, g + 1))
    assert norm_err(phi[g], ref[g]) < 1e-5
